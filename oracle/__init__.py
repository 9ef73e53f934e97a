"""FP64 CPU oracle for the D2Q9 pseudopotential LBM step (arXiv 2003.07968).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2003_07968_gb300``) never does, and shares no code with it.

The stepping code is plain C (``pplbm_oracle.c``) compiled with gcc and
loaded through ctypes; the host-side theory (Maxwell rule, Eq. PGLDR,
Lamb period, Laplace analysis) is in :mod:`oracle.theory`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pplbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_OOM = -2
ORC_ERR_NUMERIC = -4

# Carnahan-Starling constants of Eq. (CSEOS) and the text after it; G, eps and
# sigma defaults follow Sec. IV.A (G=-1, eps=1.73, sigma=1).
CS_A = 3.852462257
CS_B = 0.1304438842
CS_C = 2.785855166
CS_K = 0.01
# van der Waals in the same constants, P = k [c rho T / (1 - b rho) - a rho^2]:
# the reduced equation 8 rho T / (3 - rho) - 3 rho^2, critical point (1, 1, k)
VDW_A = 3.0
VDW_B = 1.0 / 3.0
VDW_C = 8.0 / 3.0
VDW_K = 0.01
EOS_KINDS = {"cs": 0, "vdw": 1}


class OrcParams(ctypes.Structure):
    """Mirror of ``orc_params`` in pplbm_oracle.c."""

    _fields_ = [
        ("tau", ctypes.c_double),
        ("G", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("T", ctypes.c_double),
        ("eos_a", ctypes.c_double),
        ("eos_b", ctypes.c_double),
        ("eos_c", ctypes.c_double),
        ("eos_k", ctypes.c_double),
        ("m2_trace_variant", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("mrt_rates", ctypes.c_double * 9),
        ("eos_kind", ctypes.c_int32),
    ]


def params(tau=1.0, G=-1.0, eps=1.73, sigma=1.0, T=0.8, m2_trace_variant=0,
           collision="bgk", mrt_rates=None, eos=None, eos_kind="cs") -> OrcParams:
    """Build an :class:`OrcParams`.  ``collision`` is "bgk" or "mrt"; for MRT
    the default relaxation matrix is Eq. (RM): diag(1,...,1, 1/tau, 1/tau).
    ``eos_kind`` is "cs" (Eq. CSEOS, the paper's) or "vdw" (van der Waals);
    ``eos`` = (a, b, c, k) overrides that kind's constants."""
    p = OrcParams()
    p.tau, p.G, p.eps, p.sigma, p.T = tau, G, eps, sigma, T
    if eos is None:
        eos = (CS_A, CS_B, CS_C, CS_K) if eos_kind == "cs" else (VDW_A, VDW_B, VDW_C, VDW_K)
    p.eos_a, p.eos_b, p.eos_c, p.eos_k = eos
    p.eos_kind = EOS_KINDS[eos_kind]
    p.m2_trace_variant = int(m2_trace_variant)
    p.collision = {"bgk": 0, "mrt": 1}[collision]
    rates = mrt_rates if mrt_rates is not None else [1.0] * 7 + [1.0 / tau] * 2
    for i in range(9):
        p.mrt_rates[i] = float(rates[i])
    return p


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(OrcParams)
            L.orc_eos_pressure.argtypes = [pp, ctypes.c_double]
            L.orc_eos_pressure.restype = ctypes.c_double
            L.orc_psi.argtypes = [pp, ctypes.c_double, dp]
            L.orc_psi.restype = ctypes.c_int
            L.orc_psi_field.argtypes = [pp, ctypes.c_int64, dp, dp]
            L.orc_psi_field.restype = ctypes.c_int64
            L.orc_force_moments.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_force_moments.restype = None
            L.orc_force_brute.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_force_brute.restype = None
            L.orc_init_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            L.orc_init_equilibrium.restype = None
            L.orc_step.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int64)]
            L.orc_step.restype = ctypes.c_int
            L.orc_moments.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_moments.restype = ctypes.c_int
            L.orc_mass.argtypes = [ctypes.c_int, ctypes.c_int, dp]
            L.orc_mass.restype = ctypes.c_double
            L.orc_site_terms.argtypes = [ctypes.c_double] * 5 + [dp, dp]
            L.orc_site_terms.restype = None
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_set_num_threads.restype = None
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def eos_pressure(p: OrcParams, rho: float) -> float:
    """Eq. (CSEOS)."""
    return lib().orc_eos_pressure(ctypes.byref(p), float(rho))


def psi(p: OrcParams, rho) -> np.ndarray:
    """Eq. (DED) elementwise; NaN where psi is undefined."""
    r = _f64(rho)
    out = np.empty_like(r)
    lib().orc_psi_field(ctypes.byref(p), r.size, _dp(r), _dp(out))
    return out


def force_moments(p: OrcParams, psi_field) -> tuple[np.ndarray, np.ndarray]:
    """Eq. (IFT) from a periodic psi field [ny, nx] through the psi moments."""
    ps = _f64(psi_field)
    ny, nx = ps.shape
    fx, fy = np.empty_like(ps), np.empty_like(ps)
    lib().orc_force_moments(ctypes.byref(p), nx, ny, _dp(ps), _dp(fx), _dp(fy))
    return fx, fy


def force_brute(p: OrcParams, psi_field) -> tuple[np.ndarray, np.ndarray]:
    """Eq. (Ansatz): sum_ij A_ij psi_i psi_j, on a periodic psi field [ny, nx]."""
    ps = _f64(psi_field)
    ny, nx = ps.shape
    fx, fy = np.empty_like(ps), np.empty_like(ps)
    lib().orc_force_brute(ctypes.byref(p), nx, ny, _dp(ps), _dp(fx), _dp(fy))
    return fx, fy


def init_equilibrium(rho, ux=None, uy=None) -> np.ndarray:
    """f = feq(rho, u), layout [9, ny, nx]."""
    r = _f64(rho)
    ny, nx = r.shape
    f = np.empty((9, ny, nx), dtype=np.float64)
    uxa = _f64(ux) if ux is not None else None
    uya = _f64(uy) if uy is not None else None
    lib().orc_init_equilibrium(nx, ny, _dp(r), _dp(uxa) if uxa is not None else None,
                               _dp(uya) if uya is not None else None, _dp(f))
    return f


class OracleNumericError(RuntimeError):
    pass


def step(p: OrcParams, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Advance f [9, ny, nx] (in place, and returned) by ``nsteps`` steps."""
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape[0] == 9
    _, ny, nx = f.shape
    done = ctypes.c_int64(0)
    rc = lib().orc_step(ctypes.byref(p), nx, ny, _dp(f), int(nsteps), ctypes.byref(done))
    if rc == ORC_ERR_NUMERIC:
        raise OracleNumericError(f"psi undefined after {done.value} steps")
    if rc != ORC_OK:
        raise RuntimeError(f"orc_step failed: {rc}")
    return f


def moments(p: OrcParams, f: np.ndarray) -> dict:
    """rho, force-shifted u, and force F of the state f [9, ny, nx]."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = {k: np.empty((ny, nx)) for k in ("rho", "ux", "uy", "Fx", "Fy")}
    rc = lib().orc_moments(ctypes.byref(p), nx, ny, _dp(f), _dp(out["rho"]), _dp(out["ux"]),
                           _dp(out["uy"]), _dp(out["Fx"]), _dp(out["Fy"]))
    if rc == ORC_ERR_NUMERIC:
        raise OracleNumericError("psi undefined in moments")
    return out


def mass(f: np.ndarray) -> float:
    f = _f64(f)
    _, ny, nx = f.shape
    return lib().orc_mass(nx, ny, _dp(f))


def site_terms(rho, ux, uy, Fx, Fy):
    """(feq[9], raw Guo source s[9]) at one site, Eqs. (SEDF), (GFS)."""
    feq, s = np.empty(9), np.empty(9)
    lib().orc_site_terms(float(rho), float(ux), float(uy), float(Fx), float(Fy), _dp(feq), _dp(s))
    return feq, s


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def run(p: OrcParams, rho0, nsteps: int, ux=None, uy=None) -> dict:
    """Initialise at equilibrium from ``rho0`` and run ``nsteps`` steps;
    returns the moments dict plus the final populations under ``f``."""
    f = init_equilibrium(rho0, ux, uy)
    step(p, f, nsteps)
    m = moments(p, f)
    m["f"] = f
    m["mass"] = mass(f)
    return m
