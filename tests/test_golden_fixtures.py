"""The stored oracle samples of the full-size nonlinear PB workloads
(tests/golden/*.txt, written by tests/golden/make_full_nlpb_samples.py from
the oracle's Algorithm 4) are complete and self-consistent: the sampled
indices are the generator's seeded ones plus the location of the largest
magnitude, whose value is the stated maximum, and no sample exceeds it or
the L2 norm."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _gen():
    path = os.path.join(HERE, "golden", "make_full_nlpb_samples.py")
    spec = importlib.util.spec_from_file_location("make_full_nlpb_samples", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("case", ["surface", "free"])
def test_fixture_consistent(case):
    gen = _gen()
    wl, fname, _ = gen.CASES[case]
    if not os.path.exists(os.path.join(HERE, "golden", fname)):
        pytest.fail(f"missing fixture {fname}")
    shape, stats, idx, val = gen.load(fname)
    size = int(np.prod(shape))
    seeded = gen.sample_indices(size, 20150900 + wl)
    assert np.all(np.isin(seeded, idx)) and idx.size in (seeded.size, seeded.size + 1)
    assert np.all(np.diff(idx) > 0) and idx[-1] < size
    amax = int(open(os.path.join(HERE, "golden", fname)).read().split("maxabs ")[1].split(" at ")[1].split()[0])
    assert amax in idx and abs(val[np.searchsorted(idx, amax)]) == stats["maxabs"]
    assert np.max(np.abs(val)) == stats["maxabs"] and stats["maxabs"] <= stats["l2"]
    assert np.all(np.isfinite(val)) and abs(stats["sum"]) <= np.sqrt(size) * stats["l2"]
