"""FP64 CPU oracle of the FlexRT adaptive ray-tracing step (arXiv:2409.04521).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2409_04521_gb300``) never imports it, and
this package imports nothing from the product path: the two share only the
seeded input generators in ``workloads``.

The arithmetic lives in ``flexrt_oracle.c`` (plain C, double precision,
physical cgs units, no FMA contraction); this module builds it with gcc and
wraps it with ctypes.  Every function cites the passage of the paper it
follows in the C source.

Parity pins: pix2vec, rotation, split table, traversal, chemistry and the
whole step are pinned in ``tests/test_oracle_*.py`` against closed forms,
brute force and the analytic Stromgren solution.  The temperature update
(Sec. 4.1, Eq. 12 with the Hui & Gnedin 1997 / Cen 1992 rate fits) is
checked only through limits and invariants (equilibrium, pure cooling
direction, particle-number term): it has no closed form to pin against.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flexrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXB = 8
MAXL = 13


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("z", C.c_double),
        ("nb", C.c_int32),
        ("frac", C.c_double * MAXB), ("sigma", C.c_double * MAXB), ("eheat", C.c_double * MAXB),
        ("mfp_mode", C.c_int32),
        ("lambda0_c", C.c_double), ("delta_exp", C.c_double), ("gamma_ref", C.c_double),
        ("gamma_exp", C.c_double), ("gamma_floor", C.c_double), ("xion_thr", C.c_double),
        ("nH_mean", C.c_double),
        ("l_src", C.c_int32), ("l_max", C.c_int32),
        ("n_min", C.c_double), ("eps_term", C.c_double),
        ("seed", C.c_uint64),
        ("rotate", C.c_int32), ("isothermal", C.c_int32), ("rates", C.c_int32), ("chem_iters", C.c_int32),
        ("alpha_const", C.c_double), ("x_init", C.c_double), ("T_init", C.c_double),
        ("merge", C.c_int32), ("l_merge", C.c_int32), ("n_ex", C.c_double),
        ("gamma_iters", C.c_int32), ("gen_mode", C.c_int32), ("chi", C.c_double),
        ("t_reion", C.c_double), ("alpha_pl", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.or_pix2vec.argtypes = [C.c_int, C.c_int64, P(C.c_double)]
            L.or_sm_draw.argtypes = [C.c_uint64, C.c_int32]
            L.or_sm_draw.restype = C.c_uint64
            L.or_rot_key.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
            L.or_rot_key.restype = C.c_uint64
            L.or_rotation.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int, P(C.c_double), P(C.c_int32)]
            L.or_merge_rotation.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int, P(C.c_int32)]
            L.or_direction.argtypes = [C.c_int, C.c_int64, P(C.c_int32), P(C.c_int32)]
            L.or_split_table.argtypes = [C.c_double, P(C.c_int32)]
            L.or_traverse.argtypes = [P(C.c_int64), P(C.c_int32), P(C.c_int32), P(C.c_int32),
                                      P(C.c_double), P(C.c_int)]
            L.or_alpha_B.argtypes = [C.c_double]
            L.or_alpha_B.restype = C.c_double
            L.or_alpha_A.argtypes = [C.c_double]
            L.or_alpha_A.restype = C.c_double
            L.or_pl_heat_per_ion.argtypes = [C.c_double]
            L.or_pl_heat_per_ion.restype = C.c_double
            L.or_gen_temperature.argtypes = [C.c_double] * 10
            L.or_gen_temperature.restype = C.c_double
            L.or_coll_ion.argtypes = [C.c_double]
            L.or_coll_ion.restype = C.c_double
            L.or_cooling.argtypes = [C.c_double] * 5
            L.or_cooling.restype = C.c_double
            L.or_chem_cell.argtypes = [C.c_double] * 5 + [C.c_int, C.c_double, P(C.c_double), P(C.c_double)]
            L.or_temperature.argtypes = [C.c_double] * 8
            L.or_temperature.restype = C.c_double
            L.or_create.argtypes = [P(Config), P(C.c_double)]
            L.or_create.restype = C.c_void_p
            L.or_destroy.argtypes = [C.c_void_p]
            L.or_add_sources.argtypes = [C.c_void_p, C.c_int32, P(C.c_int32), P(C.c_double)]
            L.or_step.argtypes = [C.c_void_p, C.c_double]
            L.or_get_fields.argtypes = [C.c_void_p] + [P(C.c_double)] * 4
            L.or_get_budget.argtypes = [C.c_void_p, P(C.c_double)]
            L.or_get_counts.argtypes = [C.c_void_p, P(C.c_int64)]
            L.or_get_segcount.argtypes = [C.c_void_p, P(C.c_int32)]
            L.or_get_deposits.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
            L.or_get_rays.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int64), P(C.c_int32), P(C.c_int32),
                                      P(C.c_int32), P(C.c_double), C.c_int64]
            L.or_get_rays.restype = C.c_int64
            L.or_get_rays_aux.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_int64),
                                          P(C.c_double), C.c_int64]
            L.or_get_rays_aux.restype = C.c_int64
            L.or_get_gen.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
            L.or_apply_merge.argtypes = [C.c_void_p, C.c_double, C.c_int64]
            L.or_set_rays.argtypes = [C.c_void_p, C.c_int64, C.c_int64, P(C.c_int32), P(C.c_int64), P(C.c_int32),
                                      P(C.c_int32), P(C.c_int32), P(C.c_double), P(C.c_int32), P(C.c_int32),
                                      P(C.c_int32), P(C.c_int64), P(C.c_double)]
            L.or_merge_pixel.argtypes = [C.c_int, P(C.c_int32), P(C.c_int32)]
            L.or_merge_pixel.restype = C.c_int64
            L.or_vertex_child.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int64]
            L.or_vertex_child.restype = C.c_int64
            L.or_num_emitters.argtypes = [C.c_void_p]
            L.or_num_emitters.restype = C.c_int32
            L.or_config_size.restype = C.c_int64
            assert L.or_config_size() == C.sizeof(Config), "oracle config layout mismatch"
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# --------------------------------------------------------------------------
# single functions
# --------------------------------------------------------------------------
def pix2vec(level: int, p: int) -> np.ndarray:
    """NESTED HEALPix pixel centre (Sec. 3.1, Eq. 1; Gorski et al. 2005)."""
    v = np.zeros(3)
    if lib().or_pix2vec(level, p, _p(v, C.c_double)) != 0:
        raise ValueError("bad pixel")
    return v


def splitmix_draw(key: int, i: int) -> int:
    """i-th output (0-based) of SplitMix64 started from state `key`."""
    return int(lib().or_sm_draw(key, i))


def rotation_key(seed: int, emitter: int, step: int) -> int:
    return int(lib().or_rot_key(seed, emitter, step))


def rotation(seed: int, emitter: int, step: int, rotate: bool = True):
    """Per-(emitter, step) random rotation (Sec. 3.1): (R float64[3,3], Rq int32[3,3])."""
    R = np.zeros(9)
    Rq = np.zeros(9, np.int32)
    lib().or_rotation(seed, emitter, step, int(rotate), _p(R, C.c_double), _p(Rq, C.c_int32))
    return R.reshape(3, 3), Rq.reshape(3, 3)


def merge_rotation(seed: int, cell: int, step: int, rotate: bool = True) -> np.ndarray:
    """Rotation of a cell's merge sphere (Sec. 3.3), drawn like an emitter's
    sphere with the key 2^31 + cell: Rq int32[3,3] = round(R * 2^24)."""
    Rq = np.zeros(9, np.int32)
    lib().or_merge_rotation(seed, cell, step, int(rotate), _p(Rq, C.c_int32))
    return Rq.reshape(3, 3)


def direction(level: int, p: int, Rq) -> np.ndarray:
    """Fixed-point (2^-21 cell) direction of pixel (level, p) rotated by Rq."""
    Rq = np.ascontiguousarray(np.asarray(Rq, np.int32).reshape(9))
    d = np.zeros(3, np.int32)
    if lib().or_direction(level, p, _p(Rq, C.c_int32), _p(d, C.c_int32)) != 0:
        raise ValueError("bad pixel")
    return d


def split_table(n_min: float) -> np.ndarray:
    """K[l]: whole steps after which a level-l ray splits (Sec. 3.2, Eq. 2)."""
    K = np.zeros(MAXL, np.int32)
    lib().or_split_table(n_min, _p(K, C.c_int32))
    return K


def traverse(p0, d, n):
    """Cells crossed by one step from p0 along d (fixed point); returns
    (cells int32[k,3], ds float64[k], escaped bool)."""
    p0 = np.ascontiguousarray(np.asarray(p0, np.int64))
    d = np.ascontiguousarray(np.asarray(d, np.int32))
    n = np.ascontiguousarray(np.asarray(n, np.int32))
    cells = np.zeros((4, 3), np.int32)
    ds = np.zeros(4)
    esc = C.c_int(0)
    k = lib().or_traverse(_p(p0, C.c_int64), _p(d, C.c_int32), _p(n, C.c_int32),
                          _p(cells, C.c_int32), _p(ds, C.c_double), C.byref(esc))
    if k < 0:
        raise RuntimeError("traversal produced more than 4 segments")
    return cells[:k].copy(), ds[:k].copy(), bool(esc.value)


def merge_pixel(level: int, Rq, d) -> int:
    """Pixel at `level` of the fixed-point direction d on the merge sphere
    rotated by Rq (Sec. 3.3): double-precision NESTED ang2pix of Rq^T d."""
    Rq = np.ascontiguousarray(np.asarray(Rq, np.int32).reshape(9))
    d = np.ascontiguousarray(np.asarray(d, np.int32).reshape(3))
    return int(lib().or_merge_pixel(level, _p(Rq, C.c_int32), _p(d, C.c_int32)))


def vertex_child(l_merge: int, pm: int, level: int, m: int, c: int) -> int:
    """Pixel (level + m) of child c of a merged ray of `level` centred on
    merge pixel pm of level l_merge."""
    return int(lib().or_vertex_child(l_merge, pm, level, m, c))


def alpha_B(T: float) -> float:
    return lib().or_alpha_B(T)


def alpha_A(T: float) -> float:
    """Case-A recombination coefficient (Hui & Gnedin 1997), cm^3/s."""
    return lib().or_alpha_A(T)


def pl_heat_per_ion(alpha_pl: float) -> float:
    """Mean excess energy per HI photo-ionisation of a power-law spectrum
    (index alpha_pl, cut at 4 Ryd, sigma ~ nu^-2.75), the bracket of Eq. 22, erg."""
    return lib().or_pl_heat_per_ion(alpha_pl)


def gen_temperature(T, x0, x1, yion, nH, chi, t_reion, alpha_pl, z, dt) -> float:
    """Generalized-mode temperature of a cell's ionised part after dt."""
    return lib().or_gen_temperature(T, x0, x1, yion, nH, chi, t_reion, alpha_pl, z, dt)


def coll_ion(T: float) -> float:
    return lib().or_coll_ion(T)


def cooling(T, ne, nHI, nHII, z) -> float:
    return lib().or_cooling(T, ne, nHI, nHII, z)


def chem_cell(nH, gamma, alpha, C_coll, dt, iters, y0):
    """Neutral fraction after dt and its time average (Sec. 4.1, Eq. 7-10)."""
    y1 = C.c_double()
    yb = C.c_double()
    lib().or_chem_cell(nH, gamma, alpha, C_coll, dt, iters, y0, C.byref(y1), C.byref(yb))
    return y1.value, yb.value


def temperature(T, nH, x0, x1, xbar, heat, z, dt) -> float:
    return lib().or_temperature(T, nH, x0, x1, xbar, heat, z, dt)


# --------------------------------------------------------------------------
# whole simulation
# --------------------------------------------------------------------------
class OracleSim:
    """A full FP64 simulation: emission, march, deposit, split, chemistry."""

    def __init__(self, prob):
        L = lib()
        c = Config()
        c.nx, c.ny, c.nz = prob.grid
        c.dx = prob.dx_phys_cm
        c.z = prob.redshift
        sp = prob.spectrum
        if sp.nbins > MAXB:
            raise ValueError("too many bins")
        c.nb = sp.nbins
        for b in range(sp.nbins):
            c.frac[b] = sp.frac[b]
            c.sigma[b] = sp.sigma_cm2[b]
            c.eheat[b] = sp.eheat_erg[b]
        m = prob.mfp
        c.mfp_mode = m.mode
        c.lambda0_c = m.lambda0_cm_comoving
        c.delta_exp = m.delta_exp
        c.gamma_ref = m.gamma_ref
        c.gamma_exp = m.gamma_exp
        c.gamma_floor = m.gamma_floor
        c.xion_thr = m.xion_threshold
        c.nH_mean = m.nH_mean
        o = prob.options
        c.l_src, c.l_max = o.l_src, o.l_max
        c.n_min, c.eps_term = o.n_ray_min, o.eps_term
        c.seed = o.seed
        c.rotate, c.isothermal, c.rates, c.chem_iters = int(o.rotate), int(o.isothermal), int(o.rates), o.chem_iters
        c.alpha_const, c.x_init, c.T_init = o.alpha_B_const, o.x_init, o.T_init
        c.merge = int(getattr(o, "merge", False))
        c.l_merge = int(getattr(o, "l_merge", 0))
        c.n_ex = float(getattr(o, "n_ex", 0.0))
        c.gamma_iters = int(getattr(o, "gamma_iters", 1))
        c.gen_mode = int(getattr(o, "gen_mode", False))
        c.chi = float(getattr(o, "chi", 0.0))
        c.t_reion = float(getattr(o, "t_reion", 2.0e4))
        c.alpha_pl = float(getattr(o, "alpha_pl", 1.5))
        nH = np.ascontiguousarray(prob.nH, np.float64).reshape(-1)
        self.ncell = nH.size
        self.nb = sp.nbins
        self.grid = tuple(prob.grid)
        self._h = L.or_create(C.byref(c), _p(nH, C.c_double))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        if len(prob.source_ndot):
            self.add_sources(prob.source_cells, prob.source_ndot)

    def add_sources(self, cells, ndot):
        cells = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1, 3))
        ndot = np.ascontiguousarray(np.asarray(ndot, np.float64).reshape(-1))
        r = lib().or_add_sources(self._h, len(ndot), _p(cells, C.c_int32), _p(ndot, C.c_double))
        if r != 0:
            raise ValueError("bad source")

    def step(self, dt: float):
        r = lib().or_step(self._h, dt)
        if r != 0:
            raise RuntimeError(f"oracle step failed ({r})")

    def apply_merge(self, dt: float, K: int = -1):
        """Test hook: merge the live rays as at the end of the last step (K < 0:
        floor(N_ex * N_RT) rays exempt)."""
        if lib().or_apply_merge(self._h, dt, int(K)) != 0:
            raise RuntimeError("oracle merge failed")

    def set_rays(self, step: int, r):
        """Test hook: replace the live rays by `r` (a dict as rays() returns)
        as they stand after the march of `step`."""
        n = len(r["level"])
        def a(k, t, shape=None):
            return np.ascontiguousarray(np.asarray(r[k]).astype(t).reshape(shape if shape else (n,)))
        em = np.asarray(r["emitter"]).astype(np.int64)
        merged = np.asarray(r.get("merged", np.zeros(n, bool))).astype(bool)
        em32 = np.ascontiguousarray(np.where(merged, em - (1 << 31), em).astype(np.int32))
        arrs = [a("level", np.int32), a("pixel", np.int64), em32, a("birth", np.int32), a("dir", np.int32, (n, 3)),
                a("N", np.float64, (n, self.nb)), np.ascontiguousarray(merged.astype(np.int32)),
                a("vertex", np.int32), a("A", np.int32), a("P", np.int64, (n, 3)), a("thr", np.float64)]
        cts = [C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_int32,
               C.c_int64, C.c_double]
        if lib().or_set_rays(self._h, int(step), n, *[_p(x, t) for x, t in zip(arrs, cts)]) != 0:
            raise MemoryError("oracle set_rays failed")

    def fields(self):
        out = {k: np.zeros(self.ncell) for k in ("gamma_HI", "x_HII", "T", "n_HI")}
        lib().or_get_fields(self._h, *[_p(out[k], C.c_double) for k in ("gamma_HI", "x_HII", "T", "n_HI")])
        return out

    def gen_state(self):
        """Generalized mode: (ionised volume fraction, neutral fraction inside it) per cell."""
        x = np.zeros(self.ncell)
        y = np.zeros(self.ncell)
        lib().or_get_gen(self._h, _p(x, C.c_double), _p(y, C.c_double))
        return x, y

    def budget(self):
        b = np.zeros(4)
        lib().or_get_budget(self._h, _p(b, C.c_double))
        return b

    def counts(self):
        c = np.zeros(5, np.int64)
        lib().or_get_counts(self._h, _p(c, C.c_int64))
        return dict(rays=int(c[0]), segments_last=int(c[1]), segments_total=int(c[2]),
                    step=int(c[3]), near_threshold=int(c[4]))

    def segment_counts(self):
        s = np.zeros(self.ncell, np.int32)
        lib().or_get_segcount(self._h, _p(s, C.c_int32))
        return s

    def deposits(self):
        a = np.zeros(self.ncell)
        g = np.zeros(self.ncell)
        lib().or_get_deposits(self._h, _p(a, C.c_double), _p(g, C.c_double))
        return a, g

    def rays(self):
        n = self.counts()["rays"]
        lv = np.zeros(n, np.int32)
        pix = np.zeros(n, np.int64)
        em = np.zeros(n, np.int32)
        bi = np.zeros(n, np.int32)
        d = np.zeros((n, 3), np.int32)
        N = np.zeros((n, self.nb))
        lib().or_get_rays(self._h, _p(lv, C.c_int32), _p(pix, C.c_int64), _p(em, C.c_int32),
                          _p(bi, C.c_int32), _p(d, C.c_int32), _p(N, C.c_double), n)
        kind = np.zeros(n, np.int32)
        vflag = np.zeros(n, np.int32)
        A = np.zeros(n, np.int32)
        P = np.zeros((n, 3), np.int64)
        thr = np.zeros(n)
        lib().or_get_rays_aux(self._h, _p(kind, C.c_int32), _p(vflag, C.c_int32), _p(A, C.c_int32),
                              _p(P, C.c_int64), _p(thr, C.c_double), n)
        # emitter: the emitter of a cast ray; for a merged ray 2^31 + the
        # local index of the cell it was merged in (its rotation key)
        em64 = np.where(kind == 1, em.astype(np.int64) + (1 << 31), em.astype(np.int64))
        return dict(level=lv, pixel=pix, emitter=em64, birth=bi, dir=d, N=N, merged=kind.astype(bool),
                    vertex=vflag.astype(bool), A=A, P=P, thr=thr)

    def num_emitters(self):
        return lib().or_num_emitters(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ifront_radius_cells(x_HII, x_init):
    """Sharp-boundary I-front radius from the box's ionised volume (Sec. 5.2):
    R = (3 V_ion / 4 pi)^(1/3), V_ion = sum (x - x_init)/(1 - x_init) cells."""
    v = np.sum((np.asarray(x_HII) - x_init) / (1.0 - x_init))
    return (3.0 * max(v, 0.0) / (4.0 * np.pi)) ** (1.0 / 3.0)
