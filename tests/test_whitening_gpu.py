"""Whitening-exponent study (Sec. III, Fig. 2) on the GPU against the oracle.

The paper tunes the whitening exponent between ordinary correlation (w = 0)
and phase-only correlation (w = 1) and shows, on a damaged region, a strong
match at an intermediate exponent where both ends are weak.  Stand-in:
EM-like reference patches and damaged, shifted copies (synth.damaged_pairs:
illumination gradient, a dark fold, a smeared half plane, heavy shot noise).
Every (pair, exponent) of the sweep, done as one library call, must match the
FP64 oracle at the parity tolerances.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import swim
from parity import compare, oracle_window

pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1612_04787_gb300 as swift  # noqa: E402

DEV = "cuda:0"
EXPONENTS = [0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0]


@pytest.mark.parametrize("n,count,seed", [(128, 6, 81), (256, 3, 82)])
def test_whitening_sweep_matches_the_oracle(n, count, seed):
    ref, mov, _ = synth.damaged_pairs(n, count, seed)
    res = swift.whitening_sweep(torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV), n, EXPONENTS)
    torch.cuda.synchronize()
    for e, w in enumerate(EXPONENTS):
        g = swift.decode(res[e])
        lv = swim.Level(n, w, swim.APOD_HANN, 1.0, 3.0)
        for i in range(count):
            o, tied = oracle_window(mov[i].astype(np.float64), ref[i].astype(np.float64), lv)
            compare(g, i, o, tied, n, f"w={w}")


def test_whitening_sweep_edges():
    """The sweep's rows follow the order of the exponents given (the same two
    exponents in both orders give swapped rows, bit for bit), and an empty pair
    stack gives an empty result."""
    ref, mov, _ = synth.damaged_pairs(128, 2, 83)
    tr, tm = torch.from_numpy(ref).to(DEV), torch.from_numpy(mov).to(DEV)
    a = swift.whitening_sweep(tr, tm, 128, [0.2, 0.9])
    b = swift.whitening_sweep(tr, tm, 128, [0.9, 0.2])
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[1]) and torch.equal(a[1], b[0])
    z = swift.whitening_sweep(tr[:0], tm[:0], 128, [0.5])
    assert tuple(z.shape) == (1, 0, 8)
