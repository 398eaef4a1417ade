"""GPU reverse mode against the FP64 oracle adjoint, and central finite differences at full size.

The CUDA adjoint is the transpose of the forward (2LPT of §2.1, COLA steps of §2.2, PM force of
§2.2/§2.3) with continuous CIC weights; the oracle's ``adjoint`` module is the same transpose in
FP64, itself pinned by dot-product tests and finite differences.  Bars are written per test.
"""

import numpy as np
import pytest

import cola_inputs
import oracle
from oracle import adjoint

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# oracle-sized realisations: (box, np, nmesh, ngrid)
CASES = [(128.0, 16, 32, 16), (96.0, 12, 24, 12), (150.0, 10, 30, 15), (100.0, 32, 64, 16)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1507_05329_gb300 import build
    build.build()


def ctx_for(**kw):
    from paper_1507_05329_gb300 import Context, Params
    return Context(Params(**kw))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


# ---- loss grid -----------------------------------------------------------------------------
@pytest.mark.parametrize("npd,nm,ng,amp", [(16, 32, 16, 2.0), (16, 32, 12, 5.0), (12, 24, 24, 0.7),
                                           (10, 30, 7, 9.0), (8, 8, 8, 0.0)])
def test_grid_density_matches_oracle(npd, nm, ng, amp):
    """Continuous CIC on the loss grid: FP32 weights rounded to 2^-32 against FP64 weights; a cell
    sums at most n weights, each off by < 2^-21, so |err| <= n 2^-21 ng^3 / n."""
    s = cola_inputs.random_displacements(npd, seed=npd * nm + ng, amplitude=amp)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    got = ctx.grid_density(dev(s), ng).cpu().numpy().astype(np.float64)
    ref = adjoint.grid_delta(s.astype(np.float64), npd, nm, ng)
    assert np.abs(got - ref).max() <= 2.0 ** -21 * ng ** 3
    assert abs(got.sum()) <= 1e-4 * ng ** 3   # mass conservation: mean contrast zero


def test_grid_density_is_bit_reproducible():
    s = dev(cola_inputs.random_displacements(32, seed=11, amplitude=0.4))
    ctx = ctx_for(np_side=32, nmesh=64, box=100.0)
    a = ctx.grid_density(s, 32).cpu()
    b = ctx.grid_density(s, 32).cpu()
    assert torch.equal(a, b)


@pytest.mark.parametrize("npd,nm,ng", [(16, 32, 16), (12, 24, 9)])
def test_grid_density_adjoint_matches_oracle(npd, nm, ng):
    """FP32 sums of 8 terms of size |lam| ng^4/(n nm): relative error a few 1e-7."""
    s = cola_inputs.random_displacements(npd, seed=5 + npd, amplitude=3.0)
    lam = cola_inputs.random_field((ng, ng, ng), seed=6 + ng)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    got = ctx.grid_density_adjoint(dev(s), ng, dev(lam)).cpu().numpy()
    ref = adjoint.grid_delta_adjoint(s.astype(np.float64), npd, nm, ng, lam.astype(np.float64))
    assert rel_l2(got, ref) < 1e-5


# ---- 2LPT transpose (lam_s = 0, cotangents on Psi1 and Psi2 only) -----------------------------
@pytest.mark.parametrize("box,npd,nm,ng", CASES)
def test_lpt_adjoint_matches_oracle(box, npd, nm, ng):
    """Through the autograd wrapper with gradients only on Psi1 and Psi2: FP32 FFTs of size
    np^3, relative L2 error of order 1e-6 log2(np^3); bar 1e-4."""
    from paper_1507_05329_gb300.autograd import cola_run
    w = cola_inputs.white_noise(npd, seed=31)
    lam1 = cola_inputs.random_field((3, npd ** 3), seed=32)
    lam2 = cola_inputs.random_field((3, npd ** 3), seed=33)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
    wt = dev(w).requires_grad_()
    _, _, p1, p2 = cola_run(ctx, wt)
    ((p1.double() * dev(lam1).double()).sum() + (p2.double() * dev(lam2).double()).sum()).backward()
    p = oracle.Params(box=box, np_side=npd, nmesh=nm)
    ref = adjoint.lpt_adjoint(w.astype(np.float64), lam1.astype(np.float64), lam2.astype(np.float64), p)
    assert rel_l2(wt.grad.cpu().numpy(), ref) < 1e-4


# ---- the step adjoint at the oracle's own checkpoints -------------------------------------------
def _oracle_problem(box, npd, nm, ng, seed=4, target_seed=5):
    p = oracle.Params(box=box, np_side=npd, nmesh=nm)
    w = cola_inputs.white_noise(npd, seed=seed)
    wt = cola_inputs.white_noise(npd, seed=target_seed)
    target = adjoint.grid_delta(adjoint.forward(wt.astype(np.float64), p)["s"], npd, nm, ng)
    return p, w, target


@pytest.mark.parametrize("box,npd,nm,ng", CASES[:2])
def test_adjoint_at_oracle_checkpoints(box, npd, nm, ng):
    """cola_adjoint fed the oracle's FP64 checkpoints (rounded to FP32) and final cotangent: only
    the adjoint arithmetic differs (FP32, recomputed force with 14-bit weights, 2^-20-cell
    coordinates).  Bar: relative L2 error 2e-3, correlation 0.99999."""
    p, w, target = _oracle_problem(box, npd, nm, ng)
    fwd = adjoint.forward(w.astype(np.float64), p, checkpoints=True)
    d = adjoint.grid_delta(fwd["s"], npd, nm, ng)
    lam_s = adjoint.grid_delta_adjoint(fwd["s"], npd, nm, ng, 2.0 * (d - target))
    _, ref = adjoint.gradient(w.astype(np.float64), p, ng, target)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
    ck = np.stack(fwd["checkpoints"]).astype(np.float32)
    got = ctx.adjoint(dev(w), dev(ck), dev(lam_s)).cpu().numpy()
    assert rel_l2(got, ref) < 2e-3
    assert np.corrcoef(got, ref)[0, 1] > 0.99999


# ---- end to end: GPU forward + GPU adjoint vs the oracle's gradient ------------------------------
# relative L2 bar per (particles, mesh) side: about 3x the error measured on GB300
GRADIENT_BAR = {(16, 32): 6e-4, (12, 24): 1.4e-2, (10, 30): 9e-4, (32, 64): 2.1e-3, (64, 128): 1.7e-3}


@pytest.mark.parametrize("box,npd,nm,ng", CASES + [(256.0, 64, 128, 32)])
def test_gradient_matches_oracle(box, npd, nm, ng):
    """dL/dw of L = sum (delta - delta_target)^2 through the autograd wrappers.  The GPU forward
    (fixed-point CIC, FP32) differs from the oracle's continuous-CIC FP64 forward by ~1e-4 cells,
    which moves the few particles that sit that close to a cell face to the other side of the
    one-sided weight derivative.  Bars: about 3x the errors measured on GB300 for each case (loss
    relative error up to 1.1e-5; gradient relative L2 error 1.9e-4 to 4.5e-3, the largest on the
    12^3 / 24^3 case, where a few particles sit within that distance of a cell face) and
    correlation 0.999."""
    from paper_1507_05329_gb300.autograd import cola_run, grid_density
    p, w, target = _oracle_problem(box, npd, nm, ng)
    lref, gref = adjoint.gradient(w.astype(np.float64), p, ng, target)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
    wt = dev(w).requires_grad_()
    s = cola_run(ctx, wt)[0]
    delta = grid_density(ctx, s, ng)
    loss = ((delta.double() - dev(target).double()) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(lref, rel=5e-5)
    got = wt.grad.cpu().numpy()
    print(f"gradient vs oracle ({npd}^3, {nm}^3): rel L2 {rel_l2(got, gref):.3e}, loss rel "
          f"{abs(float(loss.detach()) / lref - 1):.2e}")
    bar = GRADIENT_BAR[(npd, nm)]
    assert rel_l2(got, gref) < bar
    assert np.corrcoef(got, gref)[0, 1] > 0.999


def test_adjoint_is_linear_in_the_cotangent():
    """VJP linearity on the GPU: adjoint(a u + b v) = a adjoint(u) + b adjoint(v) to FP32 rounding."""
    npd, nm = 16, 32
    ctx = ctx_for(np_side=npd, nmesh=nm, box=128.0)
    w = dev(cola_inputs.white_noise(npd, seed=4))
    ck = ctx.run_checkpointed(w)["ckpt"]
    u = dev(cola_inputs.random_field((3, npd ** 3), seed=41))
    v = dev(cola_inputs.random_field((3, npd ** 3), seed=42))
    gu = ctx.adjoint(w, ck, u).double()
    gv = ctx.adjoint(w, ck, v).double()
    guv = ctx.adjoint(w, ck, (2.0 * u - 0.5 * v).contiguous()).double()
    err = (guv - (2.0 * gu - 0.5 * gv)).norm() / guv.norm()
    assert float(err) < 1e-5


def test_checkpointed_run_matches_plain_run():
    """The checkpointed forward is cola_run's (bit-identical s, v) and checkpoint i is s before
    step i (checkpoint 1 is the 2LPT position)."""
    npd, nm = 16, 32
    ctx = ctx_for(np_side=npd, nmesh=nm, box=128.0)
    w = dev(cola_inputs.white_noise(npd, seed=4))
    a = ctx.run_checkpointed(w)
    b = ctx.run(w, with_pk=False)
    assert torch.equal(a["s"], b["s"]) and torch.equal(a["v"], b["v"])
    s0 = ctx.ic_2lpt(w)[0]
    assert torch.equal(a["ckpt"][0], s0)
    s = s0.clone()
    v = torch.zeros_like(s)
    for i in range(1, 4):
        assert torch.equal(a["ckpt"][i - 1], s)
        ctx.step(i, s, v, a["psi1"], a["psi2"])


def test_reverse_mode_rejects_bad_arguments():
    from paper_1507_05329_gb300 import ColaError
    ctx = ctx_for(np_side=8, nmesh=16, box=64.0)
    s = torch.zeros((3, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(ColaError):
        ctx.grid_density(s, 17)   # ngrid > nmesh
    with pytest.raises(ColaError):
        ctx.grid_density(s, 0)
    r = ctx.lib.cola_adjoint(ctx._ptr, None, None, None, None, None, None, None)
    assert r == 1


# ---- full size: central finite differences ------------------------------------------------------
def test_gradient_finite_differences_full_size():
    """The differentiable workload (400 Mpc/h, 128^3 particles, 256^3 mesh, seed 4, target from
    seed 5, 64^3 loss grid): the adjoint's directional derivative along 32 random plane waves of
    the white noise (unit amplitude per site, |m_i| <= 6) against central differences of the GPU
    forward with step 1e-3 per site (a step of norm 1e-3 sqrt(n/2) = 1.45).  Smaller steps are
    dominated by the forward's quantisation (14-bit CIC weights, FP32), which makes the loss
    piecewise constant on scales of 1e-5 cells.  Bar: median relative error 3e-2 and correlation
    0.999 over the 32 directions."""
    from paper_1507_05329_gb300.autograd import cola_run, grid_density
    wl = cola_inputs.WORKLOADS["adjoint"]
    cfg = cola_inputs.ADJOINT_LOSS
    npd, ng = wl["np_side"], cfg["ngrid"]
    ctx = ctx_for(np_side=npd, nmesh=wl["nmesh"], box=wl["box"])
    w = dev(cola_inputs.white_noise(npd, seed=wl["seed"]))
    with torch.no_grad():
        tgt = grid_density(ctx, cola_run(ctx, dev(cola_inputs.white_noise(npd, seed=cfg["target_seed"])))[0],
                           ng).double()

    def loss_of(x):
        with torch.no_grad():
            return float(((grid_density(ctx, cola_run(ctx, x)[0], ng).double() - tgt) ** 2).sum())

    wt = w.clone().requires_grad_()
    loss = ((grid_density(ctx, cola_run(ctx, wt)[0], ng).double() - tgt) ** 2).sum()
    loss.backward()
    g = wt.grad.double()
    dirs = cola_inputs.plane_wave_directions(npd, cfg["fd_modes"], seed=7, mmax=cfg["fd_mmax"])
    eps = cfg["fd_eps"]
    ad, fd = [], []
    for d in dirs:
        dt = dev(d)
        ad.append(float((g * dt.double()).sum()))
        fd.append((loss_of((w + eps * dt).contiguous()) - loss_of((w - eps * dt).contiguous())) / (2 * eps))
    ad, fd = np.array(ad), np.array(fd)
    rel = np.abs(ad - fd) / np.maximum(np.abs(fd), 1e-12)
    print("fd check: median rel", np.median(rel), "max rel", rel.max(), "corr", np.corrcoef(ad, fd)[0, 1])
    assert np.median(rel) < 3e-2
    assert np.corrcoef(ad, fd)[0, 1] > 0.999
