"""B300-native batched push-rollout engine for PMBS (parallel MCTS with batched
simulation): a C-ABI CUDA library (libpmbs.so) and its thin Python binding."""
