"""Affine-warped forward and the adjoint kernels against the FP64 oracle.

Differentiation workload stand-in: a stack of EM-like sections whose cell
profiles drift slowly in z; the reference is the mean of neighbouring
sections (the paper's model, Sec. III); moving windows are resampled under
per-window affine warps (offsets up to 2 px, rotations up to 0.5 deg) whose
translations stay 0.05 px away from integers.
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


@pytest.fixture(scope="module")
def stack():
    return synth.section_stack(512, depth=5, seed=21)


def _setup(stack, n, B, seed):
    model = stack[[0, 1, 3, 4]]  # neighbours of section 2, the section itself excluded
    mov = stack[2]
    rng = np.random.default_rng(seed)
    org = synth.random_origins(B, 512, 512, n, seed=seed, margin=8)
    mo = org.copy()
    th = synth.affine_params(B, seed=seed + 1)
    return model, mov, org, mo, th, rng


def _oracle_level(lv):
    return swim.Level(lv.n, lv.whiten_exponent, swim.APOD_HANN, 1.0, lv.snr_exclusion_radius)


@pytest.mark.parametrize("n", [64, 128])
def test_warped_forward_parity(stack, n):
    model, mov, org, mo, th, _ = _setup(stack, n, 12, 5 + n)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=12)
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    g = swift.decode(plan.match(T(model), T(mov), T(org), T(mo), affine=T(th)))
    olv = _oracle_level(lv)
    for i in range(len(org)):
        m = swim.resample(mov, mo[i], n, th[i].astype(np.float64))
        r = swim.project(list(model), org[i], n)
        # the device resamples in float32: compare on its rounding of the inputs
        o, tied = oracle_window(m.astype(np.float32).astype(np.float64),
                                r.astype(np.float32).astype(np.float64), olv)
        compare(g, i, o, tied, n, f"warped n={n}")


def _grad_close(gpu, ref, rtol):
    scale = max(np.abs(ref).max(), 1e-30)
    return np.abs(gpu - ref).max() <= rtol * scale


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("w", [0.3, 0.65])
def test_backward_matches_oracle_adjoint(stack, n, w):
    B = 8
    model, mov, org, mo, th, rng = _setup(stack, n, B, 40 + n)
    gp = rng.uniform(-1, 1, B).astype(np.float32)
    gs = rng.uniform(-1, 1, B).astype(np.float32)
    lv = swift.Level(n, w, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=B)
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    g_aff, g_w = plan.backward(T(model), T(mov), T(org), T(mo), T(gp), T(gs), affine=T(th))
    torch.cuda.synchronize()
    g_aff = g_aff.cpu().numpy()
    olv = _oracle_level(lv)
    gw_ref = 0.0
    for i in range(B):
        r = swim.project(list(model), org[i], n).astype(np.float32).astype(np.float64)
        fwd, gth, gw = swim.match_backward(mov.astype(np.float64), mo[i], th[i].astype(np.float64), r, olv,
                                           float(gp[i]), float(gs[i]))
        gw_ref += gw
        assert _grad_close(g_aff[i], gth, 2e-3), (i, g_aff[i], gth)
        cos = float(np.dot(g_aff[i], gth) / (np.linalg.norm(g_aff[i]) * np.linalg.norm(gth)))
        assert cos > 0.99999, (i, cos)
    assert abs(float(g_w[0]) - gw_ref) <= 2e-3 * max(abs(gw_ref), 1e-6), (float(g_w[0]), gw_ref)


def test_autograd_function_and_descent(stack):
    """Gradients through torch.autograd, and a few descent steps on the warp
    raise the SNR-weighted peak height (loss = -sum snr * peak)."""
    n, B = 128, 16
    model, mov, org, mo, _, _ = _setup(stack, n, B, 77)
    th0 = synth.affine_params(B, seed=78, max_offset=1.5, max_rot_deg=0.4)
    lv = swift.Level(n, 0.65, "hann", 1.0, 3.0)
    plan = swift.Plan([lv], dtype="u8", max_windows=B)
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)  # noqa: E731
    ref_t, mov_t, ro, mo_t = T(model), T(mov), T(org), T(mo)
    theta = T(th0).requires_grad_(True)
    w = torch.tensor([0.65], requires_grad=True)
    peak, snr, res = swift.match_warped(plan, ref_t, mov_t, ro, mo_t, theta, w)
    loss = -(snr * peak).sum()
    loss.backward()
    ga, gw = plan.backward(ref_t, mov_t, ro, mo_t, -snr.detach(), -peak.detach(), affine=theta.detach())
    assert torch.allclose(theta.grad, ga, rtol=1e-5, atol=1e-7)
    assert w.grad is not None and w.grad.shape == (1,)
    assert torch.allclose(w.grad, gw.cpu(), rtol=1e-5, atol=1e-9)
    # descent on the translation terms only (the rotation part is small)
    start = float(loss.detach())
    th = theta.detach().clone()
    for _ in range(5):
        th.requires_grad_(True)
        pk, sn, _ = swift.match_warped(plan, ref_t, mov_t, ro, mo_t, th, w.detach())
        l = -(sn * pk).sum()
        g, = torch.autograd.grad(l, th)
        with torch.no_grad():
            step = torch.zeros_like(g)
            step[:, [2, 5]] = g[:, [2, 5]]
            th = th - 0.05 * step / (step.abs().max() + 1e-12)
    pk, sn, _ = swift.match_warped(plan, ref_t, mov_t, ro, mo_t, th, w.detach())
    assert float(-(sn * pk).sum()) < start
