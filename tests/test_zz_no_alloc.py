"""The allocation-free power-spectrum entry point (for callers that cannot call cudaMalloc, e.g.
inside a graph capture without a memory pool, or under a host framework that owns the device heap)
must give what the regular context-based entry point gives, and what the FP64 oracle gives, on two
calls in a row that share its static scratch.  It runs last so that a failure here cannot hide the
rest of the suite."""

import ctypes

import numpy as np
import pytest

import cola_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1507_05329_gb300 import build
    build.build()


def test_noalloc_matches_context_entry_point_twice():
    from paper_1507_05329_gb300 import Context, Params, binding
    cases = [(Params(box=256.0, np_side=32, nmesh=64), 64, 11),
             (Params(box=120.0, np_side=24, nmesh=48), 16, 12)]
    for p, nbins, seed in cases:
        s = torch.from_numpy(cola_inputs.random_displacements(p.np_side, seed=seed, amplitude=2.5)).cuda()
        ctx = Context(p)
        ref = ctx.power_spectrum(s, nbins)
        ctx.sync()
        ref = ref.cpu().numpy()
        for _ in range(2):
            got = binding.power_spectrum_noalloc(p, s, nbins)
            torch.cuda.synchronize()
            got = got.cpu().numpy()
            assert np.array_equal(got[2], ref[2])                       # integer mode counts
            m = ref[2] > 0
            np.testing.assert_allclose(got[0][m], ref[0][m], rtol=1e-12)  # mean |k|
            np.testing.assert_allclose(got[1][m], ref[1][m], rtol=1e-5)   # P(k), FP32 FFT
        ctx.close()


def test_noalloc_matches_the_oracle_twice():
    """P(k) of the oracle's own deposit of the same float32 displacements (§3.3 estimator): mode
    counts bit-exact, mean |k| to FP64 rounding, P to the FP32 FFT's rounding (the tolerance of the
    context entry point's parity test)."""
    from oracle import pm, power
    from paper_1507_05329_gb300 import Params, binding
    npd, nm, nb, box = 32, 64, 48, 300.0
    s_np = cola_inputs.random_displacements(npd, seed=5, amplitude=2.0)
    k, p, cnt = power.power_spectrum(pm.density_fixed(s_np, npd, nm), box, nb)
    m = cnt > 0
    s = torch.from_numpy(s_np).cuda()
    for _ in range(2):
        got = binding.power_spectrum_noalloc(Params(box=box, np_side=npd, nmesh=nm), s, nb)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert np.array_equal(got[2].astype(np.int64), cnt)
        np.testing.assert_allclose(got[0][m], k[m], rtol=1e-12)
        np.testing.assert_allclose(got[1][m], p[m], rtol=2e-5)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1507_05329_gb300 import Params, binding
    lib = binding.load_library()
    s = torch.zeros((3, 32 ** 3), device="cuda")
    pk = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    cp = Params(np_side=32, nmesh=96, box=100.0).to_c()
    st = lib.cola_power_spectrum_noalloc(ctypes.byref(cp), ctypes.c_void_p(s.data_ptr()),
                                         ctypes.c_void_p(pk.data_ptr()), 8, None)
    assert st == 1
