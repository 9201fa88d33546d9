"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Arrays are numpy; positions are uint32 fractional coordinates of shape (N, 3) on the
2^-32 grid (r = s * L / 2^32). Each function cites the equation of arXiv 2609.02694 it
evaluates; the C source states the definition term by term.
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

_LIB = None

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_dp = ct.POINTER(ct.c_double)


def lib():
    """Load (building if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ct.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_kdim_M.argtypes = [ct.c_double, ct.c_double]
        L.orc_kdim_M.restype = ct.c_int
        L.orc_kdim_table.argtypes = [ct.c_double, ct.c_double, ct.c_int, _u64p, _dp]
        L.orc_sample_k.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint32, _f64p, ct.c_double,
                                   ct.c_int, _i32p, _dp]
        L.orc_rho.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, ct.c_int, _i32p, _f64p]
        L.orc_rbe_kspace.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, ct.c_double, ct.c_double,
                                     ct.c_int, _i32p, ct.c_double, _f64p, _dp, _dp]
        L.orc_ewald_kspace.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, ct.c_double,
                                       ct.c_double, _f64p, _dp, _dp]
        L.orc_ewald_kspace_tol.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, ct.c_double,
                                           ct.c_double, ct.c_double, _f64p, _dp, _dp]
        L.orc_self_energy.argtypes = [ct.c_int64, _f64p, ct.c_double, ct.c_double]
        L.orc_self_energy.restype = ct.c_double
        L.orc_min_image_r2.argtypes = [_u32p, _u32p, _f64p, _f64p]
        L.orc_min_image_r2.restype = ct.c_double
        L.orc_real_space.argtypes = [ct.c_int64, _u32p, _f64p, _i32p, _f64p, ct.c_double,
                                     ct.c_double, ct.c_double, ct.c_int, _f64p, _f64p,
                                     ct.c_void_p, ct.c_int64, _f64p, _dp, _dp, _dp, _dp,
                                     ct.c_void_p]
        L.orc_cells.argtypes = [ct.c_int64, _u32p, _i32p, _i32p, _i64p, _i64p]
        L.orc_rbl.argtypes = [ct.c_int64, _u32p, _f64p, _i32p, _f64p, ct.c_double, ct.c_double,
                              ct.c_double, ct.c_int, ct.c_uint64, ct.c_uint64, ct.c_uint32,
                              ct.c_double, ct.c_int, _f64p, _f64p, _f64p, _dp, _dp, _dp, _dp,
                              ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.orc_rbl_rows.argtypes = [ct.c_int64, _u32p, _f64p, _i32p, _f64p, ct.c_double,
                                   ct.c_double, ct.c_double, ct.c_int, ct.c_uint64,
                                   ct.c_uint64, ct.c_uint32, ct.c_double, ct.c_int, _f64p,
                                   _f64p, _i64p, ct.c_int64, _f64p, _f64p, ct.c_void_p,
                                   ct.c_void_p, ct.c_void_p]
        L.orc_brute_coulomb.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, ct.c_double, ct.c_int,
                                        _f64p, _dp]
        L.orc_vv_drift.argtypes = [ct.c_int64, _u32p, _f64p, _f64p, _f64p, _f64p, ct.c_double,
                                   ct.c_double]
        L.orc_vv_kick.argtypes = [ct.c_int64, _f64p, _f64p, _f64p, ct.c_double, ct.c_double]
        L.orc_nh_half.argtypes = [ct.c_int64, _f64p, _f64p, ct.c_double, ct.c_double,
                                  ct.c_double, ct.c_double, ct.c_double, _f64p]
        L.orc_num_threads.restype = ct.c_int
        L.orc_set_num_threads.argtypes = [ct.c_int]
        L.orc_set_num_threads.restype = None
        for name in ("orc_kdim_table", "orc_sample_k", "orc_rho", "orc_rbe_kspace",
                     "orc_ewald_kspace", "orc_ewald_kspace_tol", "orc_real_space", "orc_cells", "orc_rbl", "orc_rbl_rows",
                     "orc_brute_coulomb", "orc_vv_drift", "orc_vv_kick", "orc_nh_half"):
            getattr(L, name).restype = ct.c_int
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _s(s):
    return np.ascontiguousarray(s, dtype=np.uint32).reshape(-1, 3)


def _f(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads for later oracle calls (timing only: no result depends on it)."""
    lib().orc_set_num_threads(int(n))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def kdim_M(L, alpha):
    return lib().orc_kdim_M(float(L), float(alpha))


def kdim_table(L, alpha, M=None):
    """Per-axis cumulative thresholds and normaliser of exp(-k^2/4 alpha) (Eq. F_long_RBE)."""
    M = kdim_M(L, alpha) if M is None else M
    T = np.zeros(2 * M + 1, np.uint64)
    Z = ct.c_double()
    _check(lib().orc_kdim_table(float(L), float(alpha), int(M), T, ct.byref(Z)), "kdim_table")
    return T, Z.value


def sample_k(seed, step, replica, box, alpha, P):
    """P importance-sampled modes m (P, 3) and the normaliser S (Eq. F_long_RBE)."""
    m = np.zeros((P, 3), np.int32)
    S = ct.c_double()
    _check(lib().orc_sample_k(int(seed), int(step), int(replica), _f(box), float(alpha),
                              int(P), m, ct.byref(S)), "sample_k")
    return m, S.value


def rho(s, q, box, m):
    """Structure factor rho(k) = sum_j q_j exp(i k.r_j) as complex128 (Eq. U_Coul_Fourier)."""
    s = _s(s)
    m = np.ascontiguousarray(m, np.int32).reshape(-1, 3)
    out = np.zeros(2 * len(m), np.float64)
    _check(lib().orc_rho(len(s), s, _f(q), _f(box), len(m), m, out), "rho")
    return out[0::2] + 1j * out[1::2]


def rbe_kspace(s, q, box, alpha, C, m, S):
    """RBE k-space force (N, 3), energy and virial on a fixed mode set (Eq. F_long_RBE)."""
    s = _s(s)
    m = np.ascontiguousarray(m, np.int32).reshape(-1, 3)
    F = np.zeros((len(s), 3), np.float64)
    U, W = ct.c_double(), ct.c_double()
    _check(lib().orc_rbe_kspace(len(s), s, _f(q), _f(box), float(alpha), float(C), len(m), m,
                                float(S), F, ct.byref(U), ct.byref(W)), "rbe_kspace")
    return F, U.value, W.value


def ewald_kspace(s, q, box, alpha, C):
    """Full Ewald k-space force, energy and virial (Eqs. U_Coul_Fourier, F_i)."""
    s = _s(s)
    F = np.zeros((len(s), 3), np.float64)
    U, W = ct.c_double(), ct.c_double()
    _check(lib().orc_ewald_kspace(len(s), s, _f(q), _f(box), float(alpha), float(C), F,
                                  ct.byref(U), ct.byref(W)), "ewald_kspace")
    return F, U.value, W.value


def ewald_kspace_tol(s, q, box, alpha, C, tol):
    """Full Ewald k-space force, energy and virial over the modes whose weight
    exp(-k^2/4 alpha) is at least tol (Eqs. U_Coul_Fourier, F_i at a stated accuracy)."""
    s = _s(s)
    F = np.zeros((len(s), 3), np.float64)
    U, W = ct.c_double(), ct.c_double()
    _check(lib().orc_ewald_kspace_tol(len(s), s, _f(q), _f(box), float(alpha), float(C),
                                      float(tol), F, ct.byref(U), ct.byref(W)),
           "ewald_kspace_tol")
    return F, U.value, W.value


def self_energy(q, alpha, C):
    q = _f(q)
    return lib().orc_self_energy(len(q), q, float(alpha), float(C))


def min_image_r2(si, sj, box):
    d = np.zeros(3, np.float64)
    r2 = lib().orc_min_image_r2(np.asarray(si, np.uint32), np.asarray(sj, np.uint32), _f(box), d)
    return r2, d


def lj_tables(eps, sig, ntypes=None):
    eps = np.atleast_1d(np.asarray(eps, np.float64))
    sig = np.atleast_1d(np.asarray(sig, np.float64))
    if ntypes is None:
        ntypes = int(round(np.sqrt(eps.size)))
    return _f(eps.reshape(-1)), _f(sig.reshape(-1)), ntypes


def real_space(s, q, types, box, alpha, rc, C, eps, sig, i_list=None):
    """Real-space erfc Coulomb + LJ forces and energies (Eqs. F_i, G_short, LJ)."""
    s = _s(s)
    N = len(s)
    eps, sig, nt = lj_tables(eps, sig)
    F = np.zeros((N, 3), np.float64)
    nbr = np.zeros(N, np.int32)
    vals = [ct.c_double() for _ in range(4)]
    if i_list is not None:
        il = np.ascontiguousarray(i_list, np.int64)
        ilp, nl = il.ctypes.data, len(il)
    else:
        il, ilp, nl = None, None, 0
    _check(lib().orc_real_space(N, s, _f(q), np.ascontiguousarray(types, np.int32), _f(box),
                                float(alpha), float(rc), float(C), nt, eps, sig, ilp, nl, F,
                                *[ct.byref(v) for v in vals], nbr.ctypes.data), "real_space")
    return dict(F=F, U_real=vals[0].value, U_lj=vals[1].value, W_real=vals[2].value,
                W_lj=vals[3].value, nbr=nbr)


def cells(s, n, within="id"):
    """Linked cells (Sec. 2.2, linked-cell reassignment and cell-wise reordering): cell of
    each particle, cell_start (ncell+1), and the ids in cell order. The paper does not fix
    the order inside a cell; within="id" orders a cell's members by id, within="x" by
    (s_x, id), the order the library and the random batch list use."""
    s = _s(s)
    n = np.ascontiguousarray(n, np.int32)
    ncell = int(np.prod(n.astype(np.int64)))
    cell_of = np.zeros(len(s), np.int32)
    cell_start = np.zeros(ncell + 1, np.int64)
    sorted_ids = np.zeros(len(s), np.int64)
    _check(lib().orc_cells(len(s), s, n, cell_of, cell_start, sorted_ids), "cells")
    if within == "x":
        for c in range(ncell):
            a, b = int(cell_start[c]), int(cell_start[c + 1])
            if b - a > 1:
                ids = sorted_ids[a:b]
                sorted_ids[a:b] = ids[np.lexsort((ids, s[ids, 0].astype(np.int64)))]
    elif within != "id":
        raise ValueError(within)
    return cell_of, cell_start, sorted_ids


def rbl(s, q, types, box, alpha, r_core, r_s, p, seed, step, replica, C, eps, sig):
    """Random batch list short-range force with the mean-force correction (Eqs. RBL, F_corr).
    Shells are enumerated over the 27 neighbour cells in (dz, dy, dx) order and inside a cell
    in ascending (s_x, id) order, the order the draws index."""
    s = _s(s)
    N = len(s)
    eps, sig, nt = lj_tables(eps, sig)
    F = np.zeros((N, 3), np.float64)
    nc = np.zeros(N, np.int32)
    ns = np.zeros(N, np.int32)
    partners = np.zeros((N, p), np.int32)
    vals = [ct.c_double() for _ in range(4)]
    _check(lib().orc_rbl(N, s, _f(q), np.ascontiguousarray(types, np.int32), _f(box),
                         float(alpha), float(r_core), float(r_s), int(p), int(seed), int(step),
                         int(replica), float(C), nt, eps, sig, F,
                         *[ct.byref(v) for v in vals], nc.ctypes.data, ns.ctypes.data,
                         partners.ctypes.data), "rbl")
    return dict(F=F, U_real=vals[0].value, U_lj=vals[1].value, W_real=vals[2].value,
                W_lj=vals[3].value, n_core=nc, n_shell=ns, partners=partners)



def rbl_rows(s, q, types, box, alpha, r_core, r_s, p, seed, step, replica, C, eps, sig,
             i_list):
    """Rows i_list of the random batch list before the mean-force correction (Eqs. Ci_Si,
    RBL): F~_i, the weighted per-row sums (U_real, U_lj, W_real, W_lj), the set sizes and
    the drawn partners, exactly as rbl computes those rows. The correction of Eq. F_corr is
    a sum over every row; a sample of rows sees it as one common offset."""
    s = _s(s)
    N = len(s)
    eps, sig, nt = lj_tables(eps, sig)
    il = np.ascontiguousarray(i_list, np.int64)
    m = len(il)
    Ft = np.zeros((m, 3), np.float64)
    u = np.zeros((m, 4), np.float64)
    nc = np.zeros(m, np.int32)
    ns = np.zeros(m, np.int32)
    partners = np.zeros((m, p), np.int32)
    _check(lib().orc_rbl_rows(N, s, _f(q), np.ascontiguousarray(types, np.int32), _f(box),
                              float(alpha), float(r_core), float(r_s), int(p), int(seed),
                              int(step), int(replica), float(C), nt, eps, sig, il, m, Ft, u,
                              nc.ctypes.data, ns.ctypes.data, partners.ctypes.data),
           "rbl_rows")
    return dict(Ft=Ft, u=u, n_core=nc, n_shell=ns, partners=partners)


def brute_coulomb(s, q, box, C, R):
    """Image-cell sum of Eq. Coul_potential for |n| <= R, in tin-foil convention."""
    s = _s(s)
    F = np.zeros((len(s), 3), np.float64)
    U = ct.c_double()
    _check(lib().orc_brute_coulomb(len(s), s, _f(q), _f(box), float(C), int(R), F,
                                   ct.byref(U)), "brute_coulomb")
    return F, U.value


def vv_drift(s, v, F, mass, box, dt, kappa):
    """First half of velocity Verlet on the fixed-point grid; updates s and v in place."""
    _check(lib().orc_vv_drift(len(s), s, v, _f(F), _f(mass), _f(box), float(dt),
                              float(kappa)), "vv_drift")


def vv_kick(v, F, mass, dt, kappa):
    _check(lib().orc_vv_kick(len(v), v, _f(F), _f(mass), float(dt), float(kappa)), "vv_kick")


def nh_half(v, mass, kappa, Nf, kT, Q, dt, xi_eta):
    """Nose-Hoover half step; v (N, 3) and xi_eta (2,) are updated in place."""
    _check(lib().orc_nh_half(len(v), v, _f(mass), float(kappa), float(Nf), float(kT), float(Q),
                             float(dt), xi_eta), "nh_half")


def total_forces(s, q, types, box, alpha, rc, C, eps, sig, m, S):
    """Total nonbonded force and energies with RBE on the given mode set (Sec. 2.1)."""
    rs = real_space(s, q, types, box, alpha, rc, C, eps, sig)
    Fk, Uk, Wk = rbe_kspace(s, q, box, alpha, C, m, S)
    Us = self_energy(q, alpha, C)
    return dict(F=rs["F"] + Fk, U_real=rs["U_real"], U_lj=rs["U_lj"], U_k=Uk, U_self=Us,
                U_total=rs["U_real"] + rs["U_lj"] + Uk - Us, W_real=rs["W_real"],
                W_lj=rs["W_lj"], W_k=Wk, nbr=rs["nbr"])


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("ct", "os", "np")]
