"""GPU friends-of-friends against the oracle (§2.3, §3.2): every link is an exact integer decision
on the deposit's fixed-point coordinates, so labels, group sizes, halo lists and halo centres of
mass (FP64 from exact integer sums, same operations) must be bit-identical."""

import numpy as np
import pytest

import cola_inputs
from oracle import cic, cola, fof

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_equal(got, ref):
    for key in ("label", "size", "halo_label", "halo_size"):
        g = got[key].cpu().numpy().astype(np.int64)
        assert np.array_equal(g, ref[key].astype(np.int64)), key
    assert got["nhalo"] == ref["halo_label"].size
    assert np.array_equal(got["halo_pos"].cpu().numpy(), ref["halo_pos"])


@pytest.fixture(scope="module")
def evolved():
    """Final positions of COLA runs (GPU forward; FoF inputs only): 32^3/64^3 and 64^3/128^3."""
    out = {}
    for npd, nm, box in ((32, 64, 128.0), (64, 128, 200.0)):
        ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
        r = ctx.run(dev(cola_inputs.white_noise(npd, seed=1)), with_pk=False)
        ctx.sync()
        out[npd] = (r["s"].cpu().numpy(), r["psi1"].cpu().numpy(), nm, box)
    return out


@pytest.mark.parametrize("npd,b,n_min", [(32, 0.2, 5), (32, 0.37, 10), (64, 0.2, 20), (64, 0.6, 1)])
def test_fof_matches_oracle_on_evolved_particles(evolved, npd, b, n_min):
    s, _, nm, box = evolved[npd]
    ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
    got = ctx.fof(dev(s), b=b, n_min=n_min)
    ctx.sync()
    ref = fof.fof(s, npd, nm, b, n_min)
    check_equal(got, ref)
    assert ref["halo_label"].size > 0


def test_fof_of_2lpt_initial_positions(evolved):
    """The 2LPT positions with the PTHalos linking length 0.37 (§3.2)."""
    _, psi1, nm, box = evolved[32]
    s = (psi1 * 2.0).astype(np.float32)
    ctx = ctx_for(np_side=32, nmesh=nm, box=box)
    got = ctx.fof(dev(s), b=0.37, n_min=8)
    ctx.sync()
    check_equal(got, fof.fof(s, 32, nm, 0.37, 8))


@pytest.mark.parametrize("b,ngroups", [(0.2, 216), (0.99, 216), (1.0, 1)])
def test_fof_unperturbed_lattice(b, ngroups):
    ctx = ctx_for(np_side=6, nmesh=12, box=60.0)
    got = ctx.fof(torch.zeros((3, 216), device="cuda"), b=b, n_min=1)
    ctx.sync()
    assert len(set(got["label"].cpu().tolist())) == ngroups
    check_equal(got, fof.fof(np.zeros((3, 216), dtype=np.float32), 6, 12, b, 1))


def test_fof_capacity_truncates_the_list_only(evolved):
    s, _, nm, box = evolved[32]
    ctx = ctx_for(np_side=32, nmesh=nm, box=box)
    full = ctx.fof(dev(s), b=0.2, n_min=2)
    part = ctx.fof(dev(s), b=0.2, n_min=2, capacity=3)
    ctx.sync()
    assert part["nhalo"] == full["nhalo"] > 3
    assert torch.equal(part["halo_label"], full["halo_label"][:3])
    assert torch.equal(part["halo_pos"], full["halo_pos"][:, :3])
    assert torch.equal(part["label"], full["label"])


def test_fof_is_bit_reproducible(evolved):
    s, _, nm, box = evolved[64]
    ctx = ctx_for(np_side=64, nmesh=nm, box=box)
    a = ctx.fof(dev(s), b=0.2, n_min=10)
    b_ = ctx.fof(dev(s), b=0.2, n_min=10)
    ctx.sync()
    for key in ("label", "size", "halo_label", "halo_size", "halo_pos"):
        assert torch.equal(a[key], b_[key]), key


def test_fof_rejects_bad_arguments():
    from paper_1507_05329_gb300 import ColaError
    ctx = ctx_for(np_side=8, nmesh=16, box=64.0)
    s = torch.zeros((3, 512), device="cuda")
    for kw in (dict(b=0.0), dict(b=-1.0), dict(n_min=0), dict(b=1e6)):
        with pytest.raises(ColaError):
            ctx.fof(s, **kw)
