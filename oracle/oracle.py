"""ctypes wrapper around the C oracle (``oracle/ppm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline / reference arm of ``bench.py``; never by the
``paper_2504_04411_gb300`` package.  It does not import that package either.

Each wrapper names the paper passage its C function restates (see the C
file's header for the list of pins that hold it to the paper).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppm_oracle.c")
_LIB = os.path.join(_HERE, "libppm_oracle.so")

NG = 12  # 2 equi-areal annuli x 6 equi-areal sectors (Sec. 6.1.1)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no implicit FMA)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")   # binary128 log-gamma (long double is binary128 on aarch64)
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_float), ("alpha", ctypes.c_float),
                ("r_min", ctypes.c_float), ("n_vm", ctypes.c_float),
                ("alpha_f", ctypes.c_double), ("rgb_test", ctypes.c_int32),
                ("vcm", ctypes.c_int32), ("i0", ctypes.c_int32),
                ("test", ctypes.c_int32), ("retrace", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, f, u32 = ctypes.c_double, ctypes.c_int, ctypes.c_float, ctypes.c_uint32
        P = ctypes.c_void_p
        _lib.oracle_betainc.restype = d
        _lib.oracle_betainc.argtypes = [d, d, d]
        _lib.oracle_f_cdf.restype = d
        _lib.oracle_f_cdf.argtypes = [d, d, d]
        _lib.oracle_f_crit.restype = d
        _lib.oracle_f_crit.argtypes = [d, d, d]
        _lib.oracle_chi2_cdf.restype = d
        _lib.oracle_chi2_cdf.argtypes = [d, d]
        _lib.oracle_chi2_crit.restype = d
        _lib.oracle_chi2_crit.argtypes = [d, d]
        _lib.oracle_chi2_counts.restype = d
        _lib.oracle_chi2_counts.argtypes = [i, P]
        _lib.oracle_anova_f.restype = d
        _lib.oracle_anova_f.argtypes = [i, d, P, P, P]
        _lib.oracle_normal_dot.restype = i
        _lib.oracle_normal_dot.argtypes = [u32, u32]
        _lib.oracle_classify.restype = i
        _lib.oracle_classify.argtypes = [P, P, P, f, P, i, u32, u32]
        _lib.oracle_radius_bound.restype = f
        _lib.oracle_radius_bound.argtypes = [f, f, i]
        _lib.oracle_shrink.restype = f
        _lib.oracle_shrink.argtypes = [f, f, f]
        _lib.oracle_lum.restype = d
        _lib.oracle_lum.argtypes = [d, d, d]
        _lib.oracle_mis_weight.restype = d
        _lib.oracle_mis_weight.argtypes = [d, d, d, d, i, d, d]
        for fn in (_lib.oracle_run, _lib.oracle_run_grid):
            fn.restype = i
            fn.argtypes = [ctypes.c_int64, P, P, P, P, P, P, i,
                           ctypes.c_int64, P, P, i, P, P, P,
                           ctypes.POINTER(_Params),
                           P, P, P, P, P, P, P, P, P, P, P]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# -- Sec. 3.2.2: F distribution -------------------------------------------
def f_cdf(d1: float, d2: float, f: float) -> float:
    return lib().oracle_f_cdf(d1, d2, f)


def f_crit(d1: float, d2: float, alpha: float) -> float:
    """(1-alpha) quantile of F(d1, d2): the critical value F_c."""
    return lib().oracle_f_crit(d1, d2, alpha)


def betainc(a: float, b: float, x: float) -> float:
    return lib().oracle_betainc(a, b, x)


# -- Sec. 3.2.3: CPPM's chi-square test of the counts -------------------------
def chi2_cdf(k: float, x: float) -> float:
    return lib().oracle_chi2_cdf(k, x)


def chi2_crit(k: float, alpha: float) -> float:
    """(1-alpha) quantile of chi^2(k): CPPM's critical value chi_c."""
    return lib().oracle_chi2_crit(k, alpha)


def chi2_counts(counts) -> float:
    """Pearson's X^2 of the counts against an even spread."""
    c = np.ascontiguousarray(counts, np.int64)
    return lib().oracle_chi2_counts(len(c), _ptr(c))


# -- Eq. (f-statistic) ------------------------------------------------------
def anova_f(groups, m: float) -> float:
    """F of a one-way ANOVA with n groups of m samples each, where group g
    lists its nonzero (or stored) samples and the rest are zeros."""
    counts = np.array([len(g) for g in groups], dtype=np.int64)
    vals = np.concatenate([np.asarray(g, dtype=np.float64) for g in groups]
                          + [np.zeros(1)])
    return lib().oracle_anova_f(len(groups), float(m), _ptr(counts),
                                _ptr(vals), None)


# -- Eq. (map-function), Sec. 3.2.1: classification ---------------------------
def normal_dot(a: int, b: int) -> int:
    return lib().oracle_normal_dot(a, b)


def classify(xh, u, v, r, xp, nq_h=None, nq_p=None) -> int:
    xh = np.ascontiguousarray(xh, np.float32)
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    xp = np.ascontiguousarray(xp, np.float32)
    use = nq_h is not None and nq_p is not None
    return lib().oracle_classify(_ptr(xh), _ptr(u), _ptr(v), np.float32(r),
                                 _ptr(xp), int(use), int(nq_h or 0),
                                 int(nq_p or 0))


# -- Eq. (radiusupdate) -------------------------------------------------------
def radius_bound(r_min: float, alpha: float, i: int) -> float:
    return lib().oracle_radius_bound(r_min, alpha, i)


def shrink(r: float, k: float, bound: float) -> float:
    return lib().oracle_shrink(r, k, bound)


# -- Sec. 5.1: the tested luminance of an RGB flux -----------------------------
def lum(R: float, G: float, B: float) -> float:
    """Rec. 709 luminance (the paper tests luminance without naming weights)."""
    return lib().oracle_lum(R, G, B)


# -- Eq. (mis-weight) ---------------------------------------------------------
def mis_weight(rho_vm_h, rho_vc_h, rho_vm_l, rho_vc_l, cos_dot, n_vm, r):
    return lib().oracle_mis_weight(rho_vm_h, rho_vc_h, rho_vm_l, rho_vc_l,
                                   int(cos_dot), n_vm, r)


@dataclass
class OracleResult:
    r: np.ndarray          # (iters+1, nh) radius used per iteration, then final
    counts: np.ndarray     # (iters, nh, 12) window counts used by the test
    S: np.ndarray          # (iters, nh, 12) window sums of psi (tested channel 0)
    Q: np.ndarray          # (iters, nh, 12) window sums of psi^2 (tested channel 0)
    F: np.ndarray          # (iters, nh)
    Fc: np.ndarray         # (iters, nh)
    reject: np.ndarray     # (iters, nh) bool
    pairs: np.ndarray      # (iters, nh) in-disk pairs of the iteration
    t: np.ndarray          # (nh,) final window length
    tau: np.ndarray        # (nh, nch) accumulated estimate sum
    Sc: np.ndarray = None  # (iters, nh, ntest, 12) window sums of psi, every tested channel
    Qc: np.ndarray = None  # (iters, nh, ntest, 12) window sums of psi^2, every tested channel
    est: np.ndarray = None  # (iters, nh, nch) each iteration's term added to tau


def run(hp: dict, photons: dict, r_init, iters: int, *, k=0.7, alpha=0.75,
        r_min=None, alpha_f=0.01, rgb_test=False, vcm=False, n_vm=None,
        i0=1, test=0, hp_iters=None, outputs=True, grid=False) -> OracleResult:
    """Run the method for ``iters`` iterations over brute-force all pairs
    (grid=True: over the photons of a sorted uniform grid's cells around each
    disk instead -- the same pairs, counts and decisions, FP64 sums added in
    cell order; the form timed as the CPU baseline).

    hp: dict with pos (nh,3), u (nh,3), v (nh,3) float32 and optional
        nq (nh,) uint32 packed normals and rho (nh,2) float32 (VCM+).
    photons: dict with pos (iters,J,3) float32, flux (iters,J) or
        (iters,J,3) float32, optional nq (iters,J) uint32, and for VCM+
        rho (iters,J,2) float32 and wq (iters,J) uint32.
    test: 0 for the ANOVA F-test, 1 for CPPM's chi-square test of the
        counts (then F holds X^2 and Fc holds chi_c).
    hp_iters: optional list of ``iters`` hit-point dicts like hp, the hit
        points traced anew for each iteration (same count and order: entry
        h is the same pixel, whose statistics carry over); hp then only
        gives the count.
    """
    if hp_iters is not None:
        if len(hp_iters) < iters:
            raise ValueError("hp_iters needs one hit-point set per iteration")
        hp = {k: np.concatenate([np.asarray(d[k]) for d in hp_iters[:iters]])
              for k in hp_iters[0] if hp_iters[0][k] is not None}
    pos = np.ascontiguousarray(hp["pos"], np.float32)
    nh = pos.shape[0]
    hu = np.ascontiguousarray(hp["u"], np.float32)
    hv = np.ascontiguousarray(hp["v"], np.float32)
    hnq = hp.get("nq")
    hnq = None if hnq is None else np.ascontiguousarray(hnq, np.uint32)
    hrho = hp.get("rho")
    hrho = None if hrho is None else np.ascontiguousarray(hrho, np.float32)
    if hp_iters is not None:
        nh //= iters
    r_init = np.ascontiguousarray(np.broadcast_to(np.float32(r_init) if np.isscalar(r_init) else r_init, (nh,)), np.float32)
    ppos = np.ascontiguousarray(photons["pos"][:iters], np.float32)
    J = ppos.shape[1]
    flux = np.ascontiguousarray(photons["flux"][:iters], np.float32)
    nch = 3 if flux.ndim == 3 else 1
    pnq = photons.get("nq")
    pnq = None if pnq is None else np.ascontiguousarray(pnq[:iters], np.uint32)
    prho = photons.get("rho")
    prho = None if prho is None else np.ascontiguousarray(prho[:iters], np.float32)
    pwq = photons.get("wq")
    pwq = None if pwq is None else np.ascontiguousarray(pwq[:iters], np.uint32)
    if r_min is None:
        r_min = 1e-3 * float(np.max(r_init)) if nh else 0.0
    prm = _Params(k=k, alpha=alpha, r_min=r_min,
                  n_vm=float(J if n_vm is None else n_vm), alpha_f=alpha_f,
                  rgb_test=int(rgb_test), vcm=int(vcm), i0=i0, test=int(test),
                  retrace=int(hp_iters is not None), pad=0)
    ntest = 3 if (rgb_test and nch == 3) else 1
    if outputs:
        o_r = np.zeros((iters + 1, nh), np.float32)
        o_c = np.zeros((iters, nh, NG), np.int32)
        o_S = np.zeros((iters, nh, ntest, NG), np.float64)
        o_Q = np.zeros((iters, nh, ntest, NG), np.float64)
        o_F = np.zeros((iters, nh), np.float64)
        o_Fc = np.zeros((iters, nh), np.float64)
        o_rej = np.zeros((iters, nh), np.uint8)
        o_pairs = np.zeros((iters, nh), np.int32)
        o_est = np.zeros((iters, nh, nch), np.float64)
    else:
        o_r = o_c = o_S = o_Q = o_F = o_Fc = o_rej = o_pairs = o_est = None
    o_t = np.zeros(nh, np.int32)
    o_tau = np.zeros((nh, nch), np.float64)
    run_fn = lib().oracle_run_grid if grid else lib().oracle_run
    rc = run_fn(nh, _ptr(pos), _ptr(hu), _ptr(hv), _ptr(hnq),
                          _ptr(hrho), _ptr(r_init), iters, J, _ptr(ppos),
                          _ptr(flux), nch, _ptr(pnq), _ptr(prho), _ptr(pwq),
                          ctypes.byref(prm), _ptr(o_r), _ptr(o_c), _ptr(o_S),
                          _ptr(o_Q), _ptr(o_F), _ptr(o_Fc), _ptr(o_rej),
                          _ptr(o_pairs), _ptr(o_t), _ptr(o_tau), _ptr(o_est))
    if rc != 0:
        raise ValueError(f"oracle_run rejected its arguments (rc={rc})")
    return OracleResult(o_r, o_c, None if o_S is None else o_S[:, :, 0, :],
                        None if o_Q is None else o_Q[:, :, 0, :], o_F, o_Fc,
                        None if o_rej is None else o_rej.astype(bool),
                        o_pairs, o_t, o_tau, Sc=o_S, Qc=o_Q, est=o_est)


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
