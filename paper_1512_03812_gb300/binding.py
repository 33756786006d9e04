"""Thin Python binding of the C ABI in ``include/schwinger.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libschwinger_gb300.so``.  There is no CPU fallback; if the library
is missing or fails to load, every call raises.

Tensor conventions (torch, on the CUDA device the lattice was created on):
  link angles q, momenta p, forces F, C, directions v: float64, shape (N, 2)
  links U64: complex128 (N, 2); U32: complex64 (N, 2)
  spinors: complex128 (N, 2) (FP64) or complex64 (N, 2) (FP32)
  per-chain values: float64 (nchains,)
where N is the total number of sites of the batch, chain c occupying rows
[offsets[c], offsets[c] + L_c T_c) with site n = x + L_c t.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

SM_OK, SM_ERR_ARG, SM_ERR_CUDA, SM_ERR_NOT_CONVERGED, SM_ERR_TIMEOUT, SM_ERR_NAN = range(6)
SM_F64, SM_F32, SM_MIXED = 0, 1, 2
PART_GAUGE, PART_FERMION, PART_FULL = 1, 2, 3
SCHEMES = {
    "leapfrog": 0,
    "five_stage": 1,
    "five_stage_fg": 2,
    "nested_leapfrog": 3,
    "nested_five_stage": 4,
    "nested_fg": 5,
    "adapted_nested_fg": 6,
    "eleven_stage": 7,
    "nested3_leapfrog": 8,
    "adapted_nested3_fg": 9,
}
THREE_LEVEL = ("nested3_leapfrog", "adapted_nested3_fg")
FG_EXACT, FG_SHIFTED = 0, 1
CG_VARIANTS = 9  # kernel variants of the chain-resident mixed CG (SM_CG_VARIANTS)
DDAGD_HEIGHTS = 8  # candidate strip heights of the streaming D^dag D (SM_DDAGD_HEIGHTS)
PART_HEAVY, PART_RATIO = 4, 8
PARTS = {"gauge": PART_GAUGE, "fermion": PART_FERMION, "full": PART_FULL, "heavy": PART_HEAVY,
         "ratio": PART_RATIO}
LAMBDA_2MN = 0.1931833275037836


class SchwingerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class NotConverged(SchwingerError):
    pass


class CgParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("algo", ctypes.c_int)]


class MdParams(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("tau", ctypes.c_double), ("n", ctypes.c_int),
                ("M", ctypes.c_int), ("lambda_", ctypes.c_double), ("fg", ctypes.c_int),
                ("merge_kicks", ctypes.c_int), ("cg", CgParams), ("tol_action", ctypes.c_double),
                ("sf_start", ctypes.c_int), ("M2", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "cg_solves", "cg_iterations", "chain_iterations", "reliable_updates", "inversions",
        "force_evals", "kernel_launches")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "sm_last_error": (ctypes.c_char_p, []),
    "sm_version": (ctypes.c_int, []),
    "sm_launch_count": (ctypes.c_longlong, []),
    "sm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "sm_profile_read": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "sm_peak_fma": (ctypes.c_int, [ctypes.c_int, _P]),
    "sm_peak_l2_read": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _P]),
    "sm_peak_smem_read": (ctypes.c_int, [_P]),
    "sm_lattice_create": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "sm_lattice_destroy": (ctypes.c_int, [_P]),
    "sm_lattice_sites": (ctypes.c_longlong, [_P]),
    "sm_lattice_check": (ctypes.c_int, [_P, _P]),
    "sm_lattice_chains": (ctypes.c_int, [_P]),
    "sm_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int]),
    "sm_lattice_set_heavy": (ctypes.c_int, [_P, ctypes.c_double]),
    "sm_debug_read": (ctypes.c_int, [_P, _P, _P]),
    "sm_workspace_bytes": (ctypes.c_size_t, [_P]),
    "sm_links": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "sm_apply_D": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "sm_apply_DdagD": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "sm_apply_DdagD_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P,
                                              _P, _P, ctypes.c_int, _P]),
    "sm_cg_solve": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(CgParams), _P,
                                   ctypes.c_size_t, _P, _P, _P]),
    "sm_autotune_cg": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(CgParams), _P,
                                      ctypes.c_size_t, _P, _P, _P]),
    "sm_set_cg_variant": (ctypes.c_int, [_P, ctypes.c_int]),
    "sm_autotune_ddagd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "sm_gauge_force": (ctypes.c_int, [_P, _P, _P, _P]),
    "sm_fermion_force": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(CgParams), _P, _P,
                                        ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_force": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(CgParams), _P, _P,
                                ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_fg_shifted_force": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(CgParams), _P, _P, ctypes.c_size_t,
                                           ctypes.POINTER(Stats), _P]),
    "sm_force_gradient": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(CgParams), _P,
                                         _P, _P, ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_hvp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.POINTER(CgParams), _P, _P,
                              ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_energies": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(CgParams), _P, _P, _P, _P,
                                   ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_md_trajectory": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(MdParams), _P,
                                        ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_md_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(MdParams), ctypes.c_double, _P,
                                  ctypes.c_size_t, ctypes.POINTER(Stats), _P]),
    "sm_hmc_graph_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(MdParams), _P,
                                           ctypes.c_size_t, ctypes.POINTER(_P), _P]),
    "sm_hmc_graph_run": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    "sm_hmc_graph_destroy": (ctypes.c_int, [_P]),
    "sm_hmc_trajectory": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(MdParams), _P,
                                         ctypes.c_size_t, _P, _P, _P, _P, _P,
                                         ctypes.POINTER(Stats), _P]),
}


def library_path() -> str:
    """The library this process loads: the bounds-checked debug build when
    the environment has SM_LIBRARY=debug, else the normal one."""
    return _build.LIB_DEBUG if os.environ.get("SM_LIBRARY") == "debug" else _build.LIB


def load() -> ctypes.CDLL:
    """Loads the CUDA library (built by ``__graft_entry__.build()`` or
    ``paper_1512_03812_gb300._build.build()``); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def _check(rc: int) -> None:
    if rc != SM_OK:
        msg = _LIB.sm_last_error().decode()
        if rc == SM_ERR_NOT_CONVERGED:
            raise NotConverged(rc, msg)
        raise SchwingerError(rc, msg)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


@dataclass
class CG:
    """CG parameters (sm_cg_params)."""
    tol: float = 1e-10
    maxit: int = 20000
    prec: str = "f64"      # "f64" or "mixed"
    delta: float = 0.1
    algo: str = "auto"     # "auto", "grid" (all chains in lockstep) or "chain" (block per chain)

    def c(self) -> CgParams:
        return CgParams(self.tol, self.maxit, {"f64": SM_F64, "mixed": SM_MIXED}[self.prec],
                        self.delta, {"auto": 0, "grid": 1, "chain": 2}[self.algo])


@dataclass
class MD:
    """Trajectory parameters (sm_md_params)."""
    scheme: str = "adapted_nested_fg"
    tau: float = 1.0
    n: int = 8
    M: int = 2
    lam: float = 1.0 / 6.0
    fg: str = "exact"       # "exact" or "shifted"
    merge_kicks: bool = True
    cg: CG = None
    tol_action: float = 0.0  # tolerance of the S_F solves of H (0: cg.tol)
    sf_start: str = "solve"  # S_F at the start of a trajectory: "solve" or "noise" (eta^dag eta)
    M2: int = 1              # three-level schemes: heavy leapfrog steps per middle block

    def c(self) -> MdParams:
        cg = self.cg or CG()
        return MdParams(SCHEMES[self.scheme], self.tau, self.n, self.M, self.lam,
                        {"exact": FG_EXACT, "shifted": FG_SHIFTED}[self.fg],
                        1 if self.merge_kicks else 0, cg.c(), self.tol_action,
                        {"solve": 0, "noise": 1}[self.sf_start], self.M2)


class Lattice:
    """A batch of independent L_c x T_c chains (sm_lattice) with couplings
    beta_c and m0_c, plus a device workspace of sm_workspace_bytes."""

    def __init__(self, L, T, beta, m0, device=None):
        lib = load()
        L = np.atleast_1d(np.asarray(L, dtype=np.int32))
        T = np.atleast_1d(np.asarray(T, dtype=np.int32))
        n = max(len(L), len(T))
        L = np.broadcast_to(L, (n,)).copy()
        T = np.broadcast_to(T, (n,)).copy()
        beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (n,)).copy()
        m0 = np.broadcast_to(np.asarray(m0, dtype=np.float64), (n,)).copy()
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            h = _P()
            _check(lib.sm_lattice_create(n, L.ctypes.data, T.ctypes.data, beta.ctypes.data,
                                         m0.ctypes.data, ctypes.byref(h)))
        self._h = h
        self.L, self.T, self.beta, self.m0 = L, T, beta, m0
        self.nchains = n
        self.N = int(lib.sm_lattice_sites(h))
        self.offsets = np.concatenate([[0], np.cumsum(L.astype(np.int64) * T)])
        self.ws_bytes = int(lib.sm_workspace_bytes(h))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.stats = Stats()

    def __del__(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.sm_lattice_destroy(self._h)
            self._h = None

    def check(self) -> int:
        """Device-side error word of this lattice (0: none), cleared; raises
        SchwingerError if a bounded device wait gave up."""
        code = ctypes.c_int()
        _check(_LIB.sm_lattice_check(self._h, ctypes.byref(code)))
        return code.value

    def set_heavy(self, dm: float):
        """Splits the fermion determinant over the masses m0 and m0 + dm
        (sm_lattice_set_heavy) and enlarges the workspace for it.  Parts
        "heavy" and "ratio" and the three-level schemes need it; their
        pseudofermion and noise tensors are then (2N, 2): phi_r / eta_r in
        the first N rows, phi_h / eta_h in the last N."""
        _check(_LIB.sm_lattice_set_heavy(self._h, float(dm)))
        self.heavy_dm = float(dm)
        self.ws_bytes = int(_LIB.sm_workspace_bytes(self._h))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def set_wait_limit(self, polls: int = -1):
        """Bound of the first wait for a tile's TMA box copies
        (sm_set_wait_limit; -1: the default)."""
        _check(_LIB.sm_set_wait_limit(self._h, int(polls)))

    # ---------------------------------------------------------- helpers --
    def field(self, dtype=torch.float64):
        return torch.empty((self.N, 2), dtype=dtype, device=self.device)

    def _ws(self):
        return self.ws.data_ptr(), self.ws_bytes

    # ------------------------------------------------------------ calls --
    def links(self, q, U64=None, U32=None):
        U64 = self.field(torch.complex128) if U64 is None else U64
        U32 = self.field(torch.complex64) if U32 is None else U32
        _check(_LIB.sm_links(self._h, _ptr(q), _ptr(U64), _ptr(U32), _stream()))
        return U64, U32

    def apply_D(self, U, psi, dagger=False, out=None):
        prec = SM_F64 if psi.dtype == torch.complex128 else SM_F32
        out = torch.empty_like(psi) if out is None else out
        _check(_LIB.sm_apply_D(self._h, _ptr(U), _ptr(psi), _ptr(out), int(dagger), prec,
                               _stream()))
        return out

    def apply_DdagD(self, U, psi, out=None):
        prec = SM_F64 if psi.dtype == torch.complex128 else SM_F32
        out = torch.empty_like(psi) if out is None else out
        _check(_LIB.sm_apply_DdagD(self._h, _ptr(U), _ptr(psi), _ptr(out), prec, *self._ws(),
                                   _stream()))
        return out

    def cg_solve(self, U64, U32, b, cg: CG, x=None):
        x = torch.empty_like(b) if x is None else x
        iters = np.zeros(self.nchains, dtype=np.int32)
        relres = np.zeros(self.nchains, dtype=np.float64)
        p = cg.c()
        _check(_LIB.sm_cg_solve(self._h, _ptr(U64), _ptr(U32), _ptr(b), _ptr(x),
                                ctypes.byref(p), *self._ws(), iters.ctypes.data,
                                relres.ctypes.data, _stream()))
        return x, iters, relres

    def autotune_cg(self, U64, U32, b, cg: CG):
        """Times the chain-resident CG kernel variants on this solve and
        keeps the fastest for this lattice (sm_autotune_cg); returns
        (variant, [ms per variant or -1])."""
        x = torch.empty_like(b)
        v = ctypes.c_int()
        ms = np.zeros(CG_VARIANTS)
        p = cg.c()
        _check(_LIB.sm_autotune_cg(self._h, _ptr(U64), _ptr(U32), _ptr(b), _ptr(x),
                                   ctypes.byref(p), *self._ws(), ctypes.byref(v), ms.ctypes.data,
                                   _stream()))
        return v.value, ms.tolist()

    def autotune_ddagd(self, U32, psi32, out=None):
        """Times the streaming D^dag D's candidate strip heights on these
        FP32 operands and keeps the fastest (sm_autotune_ddagd); returns
        (height, [(candidate height, ms per launch)]); height 0 when the
        streaming form does not serve this lattice."""
        out = torch.empty_like(psi32) if out is None else out
        h = ctypes.c_int()
        hs = np.zeros(DDAGD_HEIGHTS, dtype=np.int32)
        ms = np.zeros(DDAGD_HEIGHTS)
        _check(_LIB.sm_autotune_ddagd(self._h, _ptr(U32), _ptr(psi32), _ptr(out), ctypes.byref(h),
                                      hs.ctypes.data, ms.ctypes.data, _stream()))
        return h.value, [(int(a), float(b)) for a, b in zip(hs, ms) if a > 0]

    def hmc_graph(self, q, p0, eta, md: MD, stream=None) -> "HmcGraph":
        """Captures one HMC trajectory of every chain as a CUDA graph bound to
        these tensors (see HmcGraph)."""
        return HmcGraph(self, q, p0, eta, md, stream)

    def set_cg_variant(self, variant: int):
        """Pins the chain-resident mixed CG kernel variant (-1: default)."""
        _check(_LIB.sm_set_cg_variant(self._h, int(variant)))

    def gauge_force(self, q, F=None):
        F = self.field() if F is None else F
        _check(_LIB.sm_gauge_force(self._h, _ptr(q), _ptr(F), _stream()))
        return F

    def force(self, q, phi, part="full", cg: CG = None, F=None):
        F = self.field() if F is None else F
        p = (cg or CG()).c()
        _check(_LIB.sm_force(self._h, _ptr(q), _ptr(phi), PARTS[part], ctypes.byref(p), _ptr(F),
                             *self._ws(), ctypes.byref(self.stats), _stream()))
        return F

    def fermion_force(self, q, phi, cg: CG = None, F=None):
        F = self.field() if F is None else F
        p = (cg or CG()).c()
        _check(_LIB.sm_fermion_force(self._h, _ptr(q), _ptr(phi), ctypes.byref(p), _ptr(F),
                                     *self._ws(), ctypes.byref(self.stats), _stream()))
        return F

    def fg_shifted_force(self, q, phi, h, part="full", cg: CG = None, F=None):
        F = self.field() if F is None else F
        p = (cg or CG()).c()
        _check(_LIB.sm_fg_shifted_force(self._h, _ptr(q), _ptr(phi), PARTS[part], float(h),
                                        ctypes.byref(p), _ptr(F), *self._ws(),
                                        ctypes.byref(self.stats), _stream()))
        return F

    def force_gradient(self, q, phi, part="full", cg: CG = None, C=None, F=None):
        C = self.field() if C is None else C
        p = (cg or CG()).c()
        _check(_LIB.sm_force_gradient(self._h, _ptr(q), _ptr(phi), PARTS[part], ctypes.byref(p),
                                      _ptr(C), _ptr(F), *self._ws(), ctypes.byref(self.stats),
                                      _stream()))
        return C

    def hvp(self, q, phi, v, part="full", cg: CG = None, Hv=None):
        Hv = self.field() if Hv is None else Hv
        p = (cg or CG()).c()
        _check(_LIB.sm_hvp(self._h, _ptr(q), _ptr(phi), PARTS[part], _ptr(v), ctypes.byref(p),
                           _ptr(Hv), *self._ws(), ctypes.byref(self.stats), _stream()))
        return Hv

    def energies(self, q=None, p=None, phi=None, cg: CG = None, want=("K", "SG", "SF")):
        out = {k: torch.empty(self.nchains, dtype=torch.float64, device=self.device)
               for k in want}
        c = (cg or CG()).c()
        _check(_LIB.sm_energies(self._h, _ptr(q), _ptr(p), _ptr(phi), ctypes.byref(c),
                                _ptr(out.get("K")), _ptr(out.get("SG")), _ptr(out.get("SF")),
                                *self._ws(), ctypes.byref(self.stats), _stream()))
        return out

    def md_trajectory(self, q, p, phi, md: MD):
        m = md.c()
        _check(_LIB.sm_md_trajectory(self._h, _ptr(q), _ptr(p), _ptr(phi), ctypes.byref(m),
                                     *self._ws(), ctypes.byref(self.stats), _stream()))

    def md_step(self, q, p, phi, md: MD, h: float):
        m = md.c()
        _check(_LIB.sm_md_step(self._h, _ptr(q), _ptr(p), _ptr(phi), ctypes.byref(m), float(h),
                               *self._ws(), ctypes.byref(self.stats), _stream()))

    def hmc_trajectory(self, q, p0, eta, u, md: MD, p_out=None, q_md=None, check=True):
        """One HMC update of every chain; returns (dH, H0, accepted) as numpy
        arrays.  With check=False, chains with a non-finite Delta H or a
        failed solve are reported (rejected) instead of raising."""
        u = np.ascontiguousarray(np.broadcast_to(np.asarray(u, dtype=np.float64),
                                                 (self.nchains,)))
        dH = np.zeros(self.nchains)
        H0 = np.zeros(self.nchains)
        acc = np.zeros(self.nchains, dtype=np.int32)
        m = md.c()
        rc = _LIB.sm_hmc_trajectory(self._h, _ptr(q), _ptr(p0), _ptr(eta), u.ctypes.data,
                                    ctypes.byref(m), *self._ws(), dH.ctypes.data,
                                    H0.ctypes.data, acc.ctypes.data, _ptr(p_out), _ptr(q_md),
                                    ctypes.byref(self.stats), _stream())
        if check or rc not in (SM_ERR_NAN, SM_ERR_NOT_CONVERGED):
            _check(rc)
        return dH, H0, acc.astype(bool)


class HmcGraph:
    """A captured HMC trajectory of a lattice batch (sm_hmc_graph_*): bound to
    the tensors q (updated in place), p0 and eta (refill between runs)."""

    def __init__(self, lat: "Lattice", q, p0, eta, md: MD, stream=None):
        self.lat, self.q, self.p0, self.eta = lat, q, p0, eta  # keep the buffers alive
        self.stream = stream or torch.cuda.Stream(device=lat.device)
        self._m = md.c()
        h = _P()
        torch.cuda.current_stream(lat.device).synchronize()
        _check(_LIB.sm_hmc_graph_create(lat._h, _ptr(q), _ptr(p0), _ptr(eta), ctypes.byref(self._m),
                                        *lat._ws(), ctypes.byref(h), self.stream.cuda_stream))
        self._h = h

    def run(self, u):
        """Replays the trajectory; returns (dH, H0, accepted) like
        Lattice.hmc_trajectory(check=False)."""
        n = self.lat.nchains
        u = np.ascontiguousarray(np.broadcast_to(np.asarray(u, dtype=np.float64), (n,)))
        dH, H0 = np.zeros(n), np.zeros(n)
        acc = np.zeros(n, dtype=np.int32)
        self.stream.wait_stream(torch.cuda.current_stream(self.lat.device))
        rc = _LIB.sm_hmc_graph_run(self._h, u.ctypes.data, dH.ctypes.data, H0.ctypes.data,
                                   acc.ctypes.data, ctypes.byref(self.lat.stats),
                                   self.stream.cuda_stream)
        torch.cuda.current_stream(self.lat.device).wait_stream(self.stream)
        if rc not in (SM_ERR_NAN, SM_ERR_NOT_CONVERGED):
            _check(rc)
        return dH, H0, acc.astype(bool)

    def __del__(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.sm_hmc_graph_destroy(self._h)
            self._h = None


def apply_DdagD_noalloc(L: int, T: int, m0: float, U, psi, out=None):
    """D^dag D psi for one L x T lattice through the entry point that
    allocates nothing (sm_apply_DdagD_noalloc); for callers that cannot
    create a workspace or a lattice object.

    The C side sees only pointers and the sides L, T, so the tensors are
    checked here before anything is launched: psi of shape (L*T, 2),
    complex128 or complex64; U (links from sm_links) and out of the same
    shape and dtype; all three contiguous and on the current CUDA device.
    A mismatch raises ValueError."""
    L, T = int(L), int(T)
    if psi.dtype not in (torch.complex128, torch.complex64):
        raise ValueError(f"psi must be complex128 or complex64, got {psi.dtype}")
    out = torch.empty_like(psi) if out is None else out
    shape = (L * T, 2)
    for name, t in (("psi", psi), ("U", U), ("out", out)):
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape} for a {L} x {T} lattice, "
                             f"got {tuple(t.shape)}")
        if t.dtype != psi.dtype:
            raise ValueError(f"{name} must have psi's dtype {psi.dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t in (("psi", psi), ("U", U), ("out", out)):
        if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device, got {t.device}")
    lib = load()
    prec = SM_F64 if psi.dtype == torch.complex128 else SM_F32
    _check(lib.sm_apply_DdagD_noalloc(L, T, float(m0), _ptr(U), _ptr(psi), _ptr(out), prec,
                                      _stream()))
    return out


def profile_enable(on: bool = True) -> None:
    _check(load().sm_profile_enable(1 if on else 0))


def profile_read(reset: bool = False) -> dict:
    """Accumulated device time of the CG iteration kernels (see
    sm_profile_read)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    n, s = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().sm_profile_read(ctypes.byref(a), ctypes.byref(b), ctypes.byref(n),
                                  ctypes.byref(s), 1 if reset else 0))
    return {"iter_ms": a.value, "res_ms": b.value, "batched_iters": n.value,
            "site_iters": s.value}


def measure_peaks(l2_bytes: int = 48 << 20, l2_passes: int = 20) -> dict:
    """Measured device rates (sm_peak_*): FP64 and FP32 FMA TFLOP/s, L2 read
    GB/s over an `l2_bytes` buffer, shared-memory read GB/s."""
    lib = load()
    f64, f32, l2, smem = (ctypes.c_double() for _ in range(4))
    _check(lib.sm_peak_fma(SM_F64, ctypes.byref(f64)))
    _check(lib.sm_peak_fma(SM_F32, ctypes.byref(f32)))
    _check(lib.sm_peak_l2_read(l2_bytes, l2_passes, ctypes.byref(l2)))
    _check(lib.sm_peak_smem_read(ctypes.byref(smem)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value, "l2_read_gbs": l2.value,
            "l2_bytes": l2_bytes, "smem_read_gbs": smem.value}


def debug_read() -> dict:
    """Out-of-range indices met by the debug build since the last read
    (sm_debug_read): count, first index and the code of its place; where = -2
    in the normal build."""
    n, first, where = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    _check(load().sm_debug_read(ctypes.byref(n), ctypes.byref(first), ctypes.byref(where)))
    return {"violations": n.value, "first_index": first.value, "where": where.value}


def launch_count() -> int:
    return int(load().sm_launch_count())
