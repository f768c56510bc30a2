"""Host-side bookkeeping of bench.py and the flop model (CPU only)."""
import os

import numpy as np


def test_phase_flops_add_up_to_the_total():
    from paper_2207_06649_b300 import flops, pmbs
    rng = np.random.default_rng(0)
    ev = rng.integers(0, 10 ** 6, size=(7, len(pmbs.EVENT_NAMES))).astype(np.float64)
    total = flops.algorithmic_flops(ev, pmbs.EVENT_NAMES)
    parts = flops.flops_by_phase(ev, pmbs.EVENT_NAMES)
    assert abs(sum(parts.values()) - total) <= 1e-9 * total
    # every counted event belongs to exactly one phase
    keys = [k for ks in flops.PHASES.values() for k in ks]
    assert sorted(keys) == sorted(flops.FLOPS_PER_EVENT)


def test_kernel_hash_ignores_comments_but_not_code():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a = b"int x = 1;  // one\n\n// note\nint y = 2;\n"
    b = b"int x = 1;  // a different comment\nint y = 2;\n"
    c = b"int x = 1;\nint y = 3;\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert len(bench.kernel_source_sha()) == 16
