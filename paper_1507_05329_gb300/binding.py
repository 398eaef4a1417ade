"""Thin ctypes binding of the COLA C ABI (include/cola.h).

Argument marshalling only: every step of the method runs in the CUDA library.  Tensors are torch
CUDA tensors; the library never sees torch types, only device pointers, sizes and the stream.
There is no CPU fallback: if libcola.so is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcola.so")

STATUS = {0: "ok", 1: "invalid argument or size", 2: "device allocation failed", 3: "CUDA runtime error",
          4: "fixed-point density overflow", 5: "non-finite particle position or velocity",
          6: "internal iteration limit reached"}


class ColaError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, 'unknown status')} (cola status {status})")
        self.status = status


class CParams(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("h", ctypes.c_double), ("n_s", ctypes.c_double),
                ("sigma8", ctypes.c_double), ("box", ctypes.c_double), ("np", ctypes.c_int),
                ("nmesh", ctypes.c_int), ("nstep", ctypes.c_int), ("nlpt", ctypes.c_double),
                ("ic_mode", ctypes.c_int), ("drift_ansatz", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


@dataclasses.dataclass(frozen=True)
class Params:
    """Parameters of one realisation; field meanings as in cola_params (include/cola.h)."""

    omega_m: float = 0.27
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    box: float = 256.0
    np_side: int = 32
    nmesh: int = 64
    nstep: int = 10
    nlpt: float = -2.5
    ic_mode: int = 0
    drift_ansatz: int = 0
    seed: int = 0           # white noise of calls given white_noise=None

    @property
    def n(self) -> int:
        return self.np_side ** 3

    def to_c(self) -> CParams:
        return CParams(self.omega_m, self.h, self.n_s, self.sigma8, self.box, self.np_side, self.nmesh,
                       self.nstep, self.nlpt, self.ic_mode, self.drift_ansatz, self.seed)


_LIB = None

_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "cola_create": ([ctypes.POINTER(CParams), _VP, ctypes.POINTER(_VP)], _I),
    "cola_destroy": ([_VP], None),
    "cola_sync": ([_VP], _I),
    "cola_strerror": ([_I], ctypes.c_char_p),
    "cola_step_scalars": ([ctypes.POINTER(CParams), _I, ctypes.POINTER(_D), _I], _I),
    "cola_white_noise": ([ctypes.POINTER(CParams), _VP, _VP], _I),
    "cola_philox_words": ([ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_longlong, _VP, _VP], _I),
    "cola_linear_power": ([ctypes.POINTER(CParams), ctypes.POINTER(_D), _I, ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "cola_ic_2lpt": ([_VP, _VP, _VP, _VP, _VP, _VP], _I),
    "cola_deposit": ([_VP, _VP, _VP], _I),
    "cola_density_spectrum": ([_VP, _VP, _VP], _I),
    "cola_pm_force": ([_VP, _VP, _D, _VP], _I),
    "cola_density_spectrum_of_mesh": ([_VP, _VP, _VP], _I),
    "cola_pm_force_of_mesh": ([_VP, _VP, _D, _VP, ctypes.c_longlong, _VP], _I),
    "cola_step": ([_VP, _I, _VP, _VP, _VP, _VP], _I),
    "cola_run": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I], _I),
    "cola_run_kernel_count": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, ctypes.POINTER(ctypes.c_longlong)], _I),
    "cola_power_spectrum": ([_VP, _VP, _VP, _I], _I),
    "cola_profile_enable": ([_VP, _I], _I),
    "cola_profile_read": ([_VP, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), _I], _I),
    "cola_power_spectrum_noalloc": ([ctypes.POINTER(CParams), _VP, _VP, _I, _VP], _I),
    "cola_run_checkpointed": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "cola_adjoint": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "cola_grid_density": ([_VP, _VP, _I, _VP], _I),
    "cola_grid_density_adjoint": ([_VP, _VP, _I, _VP, _VP], _I),
    "cola_power_spectrum_ex": ([_VP, _VP, _VP, _I, _I], _I),
    "cola_snapshot": ([_VP, _I, _D, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "cola_run_snapshots": ([_VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_D), _I, _VP, _VP, _VP, _I, _I], _I),
    "cola_fof": ([_VP, _VP, _D, _I, _VP, _VP, _VP, _VP, _VP, _I, _VP], _I),
    "cola_get_schedule": ([_VP, ctypes.POINTER(_I)], _I),
    "cola_set_schedule": ([_VP, _I], _I),
    "cola_autotune": ([_VP, _VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), _I], _I),
    "cola_batch_create": ([ctypes.POINTER(CParams), _VP, _I, _I, _I, _VP, ctypes.POINTER(_VP)], _I),
    "cola_batch_run": ([_VP, _I], _I),
    "cola_batch_sync": ([_VP], _I),
    "cola_batch_tune": ([_VP, _I], _I),
    "cola_batch_info": ([_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t)], _I),
    "cola_batch_destroy": ([_VP], None),
}

PK_CIC_CORRECT = 1
SCHED_BINNED_DEPOSIT = 1
SCHED_TILE_GATHER = 2
SCHED_PIPELINED_FFT = 4
SCHED_PIPE_EPT8 = 8
SCHED_PIPELINED_GATHER = 16
SCHED_GREEN_EPT8 = 32
SCHED_C2R_EPT8 = 64
SCHED_ROWS_PIPE = 128
SCHED_BUDGET_SHIFT = 8
SCHED_R2C_EPT8 = 1024
SCHED_WIDE_TILES = 2048
SCHED_PIPE_INPLACE = 4096


class BatchIO(ctypes.Structure):
    _fields_ = [("white_noise", _VP), ("s", _VP), ("v", _VP), ("psi1", _VP), ("psi2", _VP), ("pk", _VP)]

STAGES = ["deposit", "fwd_z_r2c", "fwd_y", "green_x", "inv_y", "inv_z_c2r", "gather_kick_drift", "x_pass",
          "ic_elementwise", "pk_bins", "clear", "bin", "adjoint", "fof", "ic_fft"]


def load_library(path: str = LIB_PATH):
    """Load libcola.so (raises if it is missing: there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1507_05329_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        raise ColaError(status, what)


def step_scalars(p: Params, i: int) -> list[float]:
    """The 12 FP64 scalars of step i (i = 0: initial-condition scalars), see cola_step_scalars."""
    lib = load_library()
    out = (ctypes.c_double * 12)()
    cp = p.to_c()
    _check(lib.cola_step_scalars(ctypes.byref(cp), i, out, 12), "cola_step_scalars")
    return list(out)


def linear_power(p: Params, k) -> tuple[list[float], list[float]]:
    """The library's linear P(k) and T_BBKS(k) at a = 1 for wavenumbers k (h/Mpc), see cola_linear_power."""
    lib = load_library()
    k = [float(x) for x in k]
    kk = (ctypes.c_double * max(len(k), 1))(*k)
    pw = (ctypes.c_double * max(len(k), 1))()
    tr = (ctypes.c_double * max(len(k), 1))()
    cp = p.to_c()
    _check(lib.cola_linear_power(ctypes.byref(cp), kk, len(k), pw, tr), "cola_linear_power")
    return list(pw)[:len(k)], list(tr)[:len(k)]


def white_noise(p: Params, device=None):
    """The library's seeded white noise of p.seed on the p.np_side^3 lattice (cola_white_noise):
    a new float32 [n] tensor on `device` (default: the current CUDA device)."""
    import torch
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        out = torch.empty((p.n,), dtype=torch.float32, device=dev)
        cp = p.to_c()
        _check(lib.cola_white_noise(ctypes.byref(cp), _ptr(out, torch), ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
               "cola_white_noise")
    return out


def philox_words(seed: int, first: int, count: int, device=None):
    """Raw Philox-4x32-10 words of counters first .. first+count-1 under `seed` (cola_philox_words):
    a new int32 [count, 4] tensor holding the 32-bit words."""
    import torch
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        out = torch.empty((count, 4), dtype=torch.int32, device=dev)
        _check(lib.cola_philox_words(ctypes.c_ulonglong(seed), int(first), int(count), _ptr(out, torch),
                                     ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)), "cola_philox_words")
    return out


def power_spectrum_noalloc(p: Params, s, nbins: int = 64, stream=None):
    """P(k) of displacements s through the allocation-free entry point (no context; meshes up to
    64^3).  Returns a new [3, nbins] float64 tensor; the library itself allocates nothing."""
    import torch
    lib = load_library()
    if not s.is_cuda:
        raise ValueError("COLA tensors must live on a CUDA device")
    # the library resolves its static scratch on the current device: make that s's device
    with torch.cuda.device(s.device):
        st = stream if stream is not None else torch.cuda.current_stream(s.device)
        pk = torch.empty((3, nbins), dtype=torch.float64, device=s.device)
        cp = p.to_c()
        _check(lib.cola_power_spectrum_noalloc(ctypes.byref(cp), _ptr(s, torch, (3, p.n), torch.float32),
                                               _ptr(pk, torch), int(nbins), ctypes.c_void_p(st.cuda_stream)),
               "cola_power_spectrum_noalloc")
    return pk


def _ptr(t, torch, shape=None, dtype=None):
    if not t.is_cuda:
        raise ValueError("COLA tensors must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("COLA tensors must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One realisation's device state (cola_ctx) bound to a CUDA stream."""

    def __init__(self, params: Params, stream=None):
        import torch
        self.torch = torch
        self.p = params
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ptr = ctypes.c_void_p()
        cp = params.to_c()
        _check(self.lib.cola_create(ctypes.byref(cp), ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(self._ptr)), "cola_create")

    # -- helpers ---------------------------------------------------------------------------
    def _particles(self, t):
        return _ptr(t, self.torch, (3, self.p.n), self.torch.float32)

    def empty_particles(self):
        return self.torch.empty((3, self.p.n), dtype=self.torch.float32, device=self.device)

    @property
    def device(self):
        return self.stream.device

    def close(self):
        if self._ptr:
            self.lib.cola_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        _check(self.lib.cola_sync(self._ptr), "cola_sync")

    def _noise(self, white_noise):
        """Pointer of a caller's white noise [n], or None: the library draws the field of p.seed."""
        if white_noise is None:
            return None
        return _ptr(white_noise, self.torch, (self.p.n,), self.torch.float32)

    # -- calls -----------------------------------------------------------------------------
    def ic_2lpt(self, white_noise=None):
        wn = self._noise(white_noise)
        s, v, p1, p2 = (self.empty_particles() for _ in range(4))
        _check(self.lib.cola_ic_2lpt(self._ptr, wn, self._particles(s), self._particles(v),
                                     self._particles(p1), self._particles(p2)), "cola_ic_2lpt")
        return s, v, p1, p2

    def deposit(self, s):
        n = self.p.nmesh
        rho = self.torch.empty((n, n, n), dtype=self.torch.int64, device=self.device)
        _check(self.lib.cola_deposit(self._ptr, self._particles(s), _ptr(rho, self.torch)), "cola_deposit")
        return rho

    def density_spectrum(self, s):
        n = self.p.nmesh
        dk = self.torch.empty((n, n, n // 2 + 1, 2), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_density_spectrum(self._ptr, self._particles(s), _ptr(dk, self.torch)),
               "cola_density_spectrum")
        return dk

    def density_spectrum_of_mesh(self, rho):
        """cola_density_spectrum_of_mesh: forward spectrum [N, N, N/2+1, 2] of a given fixed-point mesh."""
        n = self.p.nmesh
        _ptr(rho, self.torch, (n, n, n), self.torch.int64)
        dk = self.torch.empty((n, n, n // 2 + 1, 2), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_density_spectrum_of_mesh(self._ptr, _ptr(rho, self.torch), _ptr(dk, self.torch)),
               "cola_density_spectrum_of_mesh")
        return dk

    def pm_force_of_mesh(self, rho, a: float, cells):
        """cola_pm_force_of_mesh: the force components [3, m] at mesh cells (int64 flat indices)."""
        n = self.p.nmesh
        _ptr(rho, self.torch, (n, n, n), self.torch.int64)
        m = int(cells.numel())
        if m and (int(cells.min()) < 0 or int(cells.max()) >= n ** 3):
            raise ValueError("cells must lie in [0, N^3)")
        out = self.torch.empty((3, m), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_pm_force_of_mesh(self._ptr, _ptr(rho, self.torch), float(a),
                                              _ptr(cells, self.torch, (m,), self.torch.int64), m, _ptr(out, self.torch)),
               "cola_pm_force_of_mesh")
        return out

    def pm_force(self, s, a: float):
        f = self.empty_particles()
        _check(self.lib.cola_pm_force(self._ptr, self._particles(s), float(a), self._particles(f)),
               "cola_pm_force")
        return f

    def step(self, i: int, s, v, psi1, psi2):
        _check(self.lib.cola_step(self._ptr, int(i), self._particles(s), self._particles(v),
                                  self._particles(psi1), self._particles(psi2)), "cola_step")

    def profile(self, on: bool = True):
        """Start (reset) or stop CUDA-event timing of every library launch on this stream."""
        _check(self.lib.cola_profile_enable(self._ptr, 1 if on else 0), "cola_profile_enable")

    def profile_read(self) -> dict:
        """{stage: (total ms, launches)} since the last profile(True); synchronises the stream."""
        ms = (ctypes.c_double * len(STAGES))()
        cnt = (ctypes.c_longlong * len(STAGES))()
        r = self.lib.cola_profile_read(self._ptr, ms, cnt, len(STAGES))
        if r < 0:
            raise ColaError(-r, "cola_profile_read")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES)}

    def power_spectrum(self, s, nbins: int = 64):
        pk = self.torch.empty((3, nbins), dtype=self.torch.float64, device=self.device)
        _check(self.lib.cola_power_spectrum(self._ptr, self._particles(s), _ptr(pk, self.torch), int(nbins)),
               "cola_power_spectrum")
        return pk

    def power_spectrum_ex(self, s, nbins: int = 64, cic_correct: bool = False):
        """cola_power_spectrum_ex: P(k), optionally CIC-window/alias corrected and shot-noise subtracted."""
        pk = self.torch.empty((3, nbins), dtype=self.torch.float64, device=self.device)
        _check(self.lib.cola_power_spectrum_ex(self._ptr, self._particles(s), _ptr(pk, self.torch), int(nbins),
                                               PK_CIC_CORRECT if cic_correct else 0), "cola_power_spectrum_ex")
        return pk

    def snapshot(self, i: int, a_snap: float, s, v, psi1, psi2, with_velocity: bool = True):
        """cola_snapshot after step i: returns (s at a_snap, canonical v at a_snap or None)."""
        so = self.empty_particles()
        vo = self.empty_particles() if with_velocity else None
        _check(self.lib.cola_snapshot(self._ptr, int(i), float(a_snap), self._particles(s), self._particles(v),
                                      self._particles(psi1), self._particles(psi2), self._particles(so),
                                      self._particles(vo) if vo is not None else None), "cola_snapshot")
        return so, vo

    def run_snapshots(self, white_noise, a_snap, nbins: int = 64, with_pk: bool = True, cic_correct: bool = False):
        """cola_run_snapshots: dict(s, v, psi1, psi2, s_snap [k,3,n], v_snap, pk_snap [k,3,nbins])."""
        wn = self._noise(white_noise)
        k = len(a_snap)
        s, v, p1, p2 = (self.empty_particles() for _ in range(4))
        ss = self.torch.empty((k, 3, self.p.n), dtype=self.torch.float32, device=self.device)
        vs = self.torch.empty((k, 3, self.p.n), dtype=self.torch.float32, device=self.device)
        pk = self.torch.empty((k, 3, nbins), dtype=self.torch.float64, device=self.device) if with_pk else None
        arr = (ctypes.c_double * k)(*[float(a) for a in a_snap])
        _check(self.lib.cola_run_snapshots(self._ptr, wn, self._particles(s), self._particles(v),
                                           self._particles(p1), self._particles(p2), arr, k, _ptr(ss, self.torch),
                                           _ptr(vs, self.torch), _ptr(pk, self.torch) if with_pk else None,
                                           int(nbins), PK_CIC_CORRECT if cic_correct else 0), "cola_run_snapshots")
        return dict(s=s, v=v, psi1=p1, psi2=p2, s_snap=ss, v_snap=vs, pk_snap=pk)

    def run(self, white_noise=None, nbins: int = 64, with_pk: bool = True, out: dict | None = None):
        """A whole realisation (cola_run).  ``out`` may hold preallocated s, v, psi1, psi2, pk tensors."""
        wn = self._noise(white_noise)
        if out is None:
            s, v, p1, p2 = (self.empty_particles() for _ in range(4))
            pk = self.torch.empty((3, nbins), dtype=self.torch.float64, device=self.device) if with_pk else None
        else:
            s, v, p1, p2, pk = out["s"], out["v"], out["psi1"], out["psi2"], out.get("pk")
            if with_pk:
                _ptr(pk, self.torch, (3, nbins), self.torch.float64)
        _check(self.lib.cola_run(self._ptr, wn, self._particles(s), self._particles(v), self._particles(p1),
                                 self._particles(p2), _ptr(pk, self.torch) if with_pk else None, int(nbins)),
               "cola_run")
        return dict(s=s, v=v, psi1=p1, psi2=p2, pk=pk)

    def run_kernel_count(self, white_noise=None, nbins: int = 64, with_pk: bool = True, out: dict | None = None) -> int:
        """Kernels one ``run`` with these arguments launches (cola_run_kernel_count: captured, counted,
        not executed).  Call after one ``run`` with the same nbins."""
        wn = self._noise(white_noise)
        if out is None:
            s, v, p1, p2 = (self.empty_particles() for _ in range(4))
            pk = self.torch.empty((3, nbins), dtype=self.torch.float64, device=self.device) if with_pk else None
        else:
            s, v, p1, p2, pk = out["s"], out["v"], out["psi1"], out["psi2"], out.get("pk")
        k = ctypes.c_longlong()
        _check(self.lib.cola_run_kernel_count(self._ptr, wn, self._particles(s), self._particles(v),
                                              self._particles(p1), self._particles(p2),
                                              _ptr(pk, self.torch) if with_pk else None, int(nbins),
                                              ctypes.byref(k)), "cola_run_kernel_count")
        return int(k.value)

    # -- reverse mode ----------------------------------------------------------------------
    def run_checkpointed(self, white_noise=None):
        """cola_run_checkpointed: returns dict(s, v, psi1, psi2, ckpt) with ckpt [nstep, 3, n]."""
        wn = self._noise(white_noise)
        s, v, p1, p2 = (self.empty_particles() for _ in range(4))
        ck = self.torch.empty((self.p.nstep, 3, self.p.n), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_run_checkpointed(self._ptr, wn, self._particles(s), self._particles(v),
                                              self._particles(p1), self._particles(p2), _ptr(ck, self.torch)),
               "cola_run_checkpointed")
        return dict(s=s, v=v, psi1=p1, psi2=p2, ckpt=ck)

    def adjoint(self, white_noise, ckpt, lam_s, lam_v=None, lam_psi1=None, lam_psi2=None):
        """cola_adjoint: dL/d(white noise) [n] from the cotangents of the final s (and optionally
        v_res, Psi1, Psi2)."""
        wn = self._noise(white_noise)
        ck = _ptr(ckpt, self.torch, (self.p.nstep, 3, self.p.n), self.torch.float32)
        opt = [None if t is None else self._particles(t) for t in (lam_v, lam_psi1, lam_psi2)]
        out = self.torch.empty((self.p.n,), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_adjoint(self._ptr, wn, ck, self._particles(lam_s), *opt, _ptr(out, self.torch)),
               "cola_adjoint")
        return out

    def grid_density(self, s, ngrid: int):
        """cola_grid_density: CIC density contrast [ngrid, ngrid, ngrid] of the particles."""
        d = self.torch.empty((ngrid, ngrid, ngrid), dtype=self.torch.float32, device=self.device)
        _check(self.lib.cola_grid_density(self._ptr, self._particles(s), int(ngrid), _ptr(d, self.torch)),
               "cola_grid_density")
        return d

    def grid_density_adjoint(self, s, ngrid: int, lam_delta):
        """cola_grid_density_adjoint: d(sum lam_delta delta)/ds [3, n]."""
        ld = _ptr(lam_delta, self.torch, (ngrid, ngrid, ngrid), self.torch.float32)
        out = self.empty_particles()
        _check(self.lib.cola_grid_density_adjoint(self._ptr, self._particles(s), int(ngrid), ld,
                                                  self._particles(out)), "cola_grid_density_adjoint")
        return out

    # -- friends-of-friends ----------------------------------------------------------------
    def fof(self, s, b: float = 0.2, n_min: int = 20, capacity: int | None = None):
        """cola_fof: dict(label [n], size [n], halo_label [h], halo_size [h], halo_pos [3, h], nhalo)."""
        t = self.torch
        n = self.p.n
        cap = n if capacity is None else int(capacity)
        label = t.empty(n, dtype=t.int32, device=self.device)
        size = t.empty(n, dtype=t.int32, device=self.device)
        hl = t.empty(max(cap, 1), dtype=t.int32, device=self.device)
        hs = t.empty(max(cap, 1), dtype=t.int32, device=self.device)
        hp = t.empty((3, max(cap, 1)), dtype=t.float64, device=self.device)
        nh = t.zeros(4, dtype=t.int32, device=self.device)
        _check(self.lib.cola_fof(self._ptr, self._particles(s), float(b), int(n_min), _ptr(label, t), _ptr(size, t),
                                 _ptr(hl, t), _ptr(hs, t), _ptr(hp, t), cap, _ptr(nh, t)), "cola_fof")
        nhalo = int(nh[0])
        k = min(nhalo, cap)
        return dict(label=label, size=size, halo_label=hl[:k], halo_size=hs[:k], halo_pos=hp[:, :k], nhalo=nhalo)

    # -- execution schedule ----------------------------------------------------------------
    @property
    def schedule(self) -> int:
        out = ctypes.c_int()
        _check(self.lib.cola_get_schedule(self._ptr, ctypes.byref(out)), "cola_get_schedule")
        return out.value

    @schedule.setter
    def schedule(self, value: int):
        _check(self.lib.cola_set_schedule(self._ptr, int(value)), "cola_set_schedule")

    def autotune(self, s, reps: int = 3):
        """cola_autotune at displacements s: returns (best schedule, {timed schedule: ms})."""
        best = ctypes.c_int()
        cap = 256
        sch = (ctypes.c_int * cap)()
        ms = (ctypes.c_double * cap)()
        r = self.lib.cola_autotune(self._ptr, self._particles(s), int(reps), ctypes.byref(best), sch, ms, cap)
        if r < 0:
            raise ColaError(-r, "cola_autotune")
        return best.value, {sch[i]: ms[i] for i in range(min(r, cap))}

    def _schedule_ok(self, sc: int) -> bool:
        keep = self.schedule
        ok = self.lib.cola_set_schedule(self._ptr, sc) == 0
        self.lib.cola_set_schedule(self._ptr, keep)
        return ok


class Batch:
    """Many realisations run as one launch sequence over `nstreams` lanes, optionally replayed from
    one CUDA graph (cola_batch_*).  Buffers are allocated here (torch) and fixed for the batch's
    lifetime; results are read from ``outputs[i]``."""

    def __init__(self, params: list, white_noise: list, nbins: int = 64, nstreams: int = 8, stream=None):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.params = list(params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        dev = self.stream.device
        self.outputs = []
        ios = (BatchIO * len(params))()
        cps = (CParams * len(params))()
        for i, (p, wn) in enumerate(zip(params, white_noise)):
            if wn is not None:   # None: the library draws the field of p.seed
                _ptr(wn, torch, (p.n,), torch.float32)
            o = {k: torch.empty((3, p.n), dtype=torch.float32, device=dev) for k in ("s", "v", "psi1", "psi2")}
            o["pk"] = torch.empty((3, nbins), dtype=torch.float64, device=dev)
            o["white_noise"] = wn
            self.outputs.append(o)
            ios[i] = BatchIO(wn.data_ptr() if wn is not None else None, o["s"].data_ptr(), o["v"].data_ptr(), o["psi1"].data_ptr(),
                             o["psi2"].data_ptr(), o["pk"].data_ptr())
            cps[i] = p.to_c()
        self._ptr = ctypes.c_void_p()
        _check(self.lib.cola_batch_create(cps, ios, len(params), int(nbins), int(nstreams),
                                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ptr)),
               "cola_batch_create")

    def run(self, use_graph: bool = True):
        _check(self.lib.cola_batch_run(self._ptr, 1 if use_graph else 0), "cola_batch_run")

    def sync(self):
        _check(self.lib.cola_batch_sync(self._ptr), "cola_batch_sync")

    def tune(self, reps: int = 3):
        _check(self.lib.cola_batch_tune(self._ptr, int(reps)), "cola_batch_tune")

    def info(self, i: int) -> dict:
        lane, sched, nodes = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(self.lib.cola_batch_info(self._ptr, int(i), ctypes.byref(lane), ctypes.byref(sched),
                                        ctypes.byref(nodes)), "cola_batch_info")
        return dict(lane=lane.value, schedule=sched.value, graph_nodes=nodes.value)

    def close(self):
        if self._ptr:
            self.lib.cola_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
