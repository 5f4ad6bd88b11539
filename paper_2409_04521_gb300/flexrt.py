"""ctypes binding of libflexrt (include/flexrt.h): argument marshalling only.

Every step of the RT method runs in the library's CUDA kernels.  There is no
CPU fallback: if the library cannot be loaded, or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FLEXRT_OK = 0
STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CAPACITY", 4: "CUDA", 5: "TIMEOUT", 6: "STATE"}
MAX_BINS = 8


class FlexRTError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"flexrt status {STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class Box(C.Structure):
    _fields_ = [("box_cm_comoving", C.c_double), ("redshift", C.c_double)]


class Spectrum(C.Structure):
    _fields_ = [("nbins", C.c_int32), ("frac", C.POINTER(C.c_double)), ("sigma_cm2", C.POINTER(C.c_double)),
                ("eheat_erg", C.POINTER(C.c_double))]


class Mfp(C.Structure):
    _fields_ = [("mode", C.c_int32), ("lambda0_cm_comoving", C.c_double), ("delta_exp", C.c_double),
                ("gamma_ref", C.c_double), ("gamma_exp", C.c_double), ("gamma_floor", C.c_double),
                ("xion_threshold", C.c_double), ("nH_mean", C.c_double)]


class Options(C.Structure):
    _fields_ = [("l_src", C.c_int32), ("l_max", C.c_int32), ("n_ray_min", C.c_double), ("eps_term", C.c_double),
                ("seed", C.c_uint64), ("rotate", C.c_int32), ("isothermal", C.c_int32), ("rates", C.c_int32),
                ("chem_iters", C.c_int32), ("alpha_B_const", C.c_double), ("x_init", C.c_double),
                ("T_init", C.c_double), ("ray_capacity", C.c_int64), ("keep_diagnostics", C.c_int32),
                ("cuda_stream", C.c_void_p), ("merge", C.c_int32), ("l_merge", C.c_int32), ("n_ex", C.c_double),
                ("gamma_iters", C.c_int32), ("gen_mode", C.c_int32), ("chi", C.c_double),
                ("t_reion", C.c_double), ("alpha_pl", C.c_double), ("device_bytes_max", C.c_int64)]


class BatchConfig(C.Structure):
    _fields_ = [("max_sims", C.c_int32), ("max_grid", C.c_int32), ("nbins", C.c_int32), ("n_ray_min", C.c_double),
                ("ray_capacity", C.c_int64), ("cell_capacity", C.c_int64), ("emitter_capacity", C.c_int32),
                ("keep_diagnostics", C.c_int32), ("use_graph", C.c_int32), ("cuda_stream", C.c_void_p),
                ("merge_l_max", C.c_int32), ("gen_capable", C.c_int32), ("device_bytes_max", C.c_int64)]


class ProbeRays(C.Structure):
    _fields_ = [("pixlev", C.POINTER(C.c_uint32)), ("emitter", C.POINTER(C.c_uint32)),
                ("birth", C.POINTER(C.c_int32)), ("dir", C.POINTER(C.c_int32)), ("photons", C.POINTER(C.c_float)),
                ("pos", C.POINTER(C.c_int32)), ("aux", C.POINTER(C.c_uint32)), ("thr", C.POINTER(C.c_float))]


class MergeProbe(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nbins", C.c_int32),
                ("l_src", C.c_int32), ("l_max", C.c_int32), ("l_merge", C.c_int32), ("k_ex", C.c_int64),
                ("seed", C.c_uint64), ("rotate", C.c_int32), ("step", C.c_int32), ("eps_term", C.c_float),
                ("n_emitters", C.c_int32), ("emitter_cell", C.POINTER(C.c_int32)),
                ("emitter_n0", C.POINTER(C.c_float))]


class Fields(C.Structure):
    _fields_ = [("gamma_HI", C.POINTER(C.c_double)), ("x_HII", C.POINTER(C.c_double)),
                ("T", C.POINTER(C.c_double)), ("n_HI", C.POINTER(C.c_double))]


def library_path() -> str:
    return _build.SO


def lib():
    """Load libflexrt (building it if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            P = C.POINTER
            vp = C.c_void_p
            L.flexrt_default_options.argtypes = [P(Options)]
            L.flexrt_create.argtypes = [P(Grid), P(Box), P(C.c_double), P(Mfp), P(Spectrum), P(Options), P(vp)]
            L.flexrt_add_sources.argtypes = [vp, C.c_int32, P(C.c_int32), P(C.c_double)]
            L.flexrt_step.argtypes = [vp, C.c_double]
            L.flexrt_step_stage.argtypes = [vp, C.c_double, C.c_int32]
            L.flexrt_sync.argtypes = [vp]
            L.flexrt_reset.argtypes = [vp]
            L.flexrt_get_fields.argtypes = [vp, P(Fields)]
            L.flexrt_get_budget.argtypes = [vp, P(C.c_double)]
            L.flexrt_get_screen_excess.argtypes = [vp, P(C.c_double)]
            L.flexrt_get_counts.argtypes = [vp, P(C.c_int64)]
            L.flexrt_get_segment_counts.argtypes = [vp, P(C.c_int32)]
            L.flexrt_get_rays.argtypes = [vp, C.c_int64, P(C.c_int32), P(C.c_int64), P(C.c_int32), P(C.c_int32),
                                          P(C.c_int32), P(C.c_double), P(C.c_int64)]
            L.flexrt_get_ionized_volume.argtypes = [vp, P(C.c_double)]
            L.flexrt_batch_get_ionized_volume.argtypes = [vp, C.c_int32, P(C.c_double)]
            L.flexrt_get_rays_merged.argtypes = [vp, C.c_int64, P(C.c_int32), P(C.c_int32), P(C.c_int32),
                                                 P(C.c_int64), P(C.c_double), P(C.c_int64)]
            L.flexrt_profile.argtypes = [vp, C.c_int32]
            L.flexrt_save_state.argtypes = [vp, vp, C.c_int64, P(C.c_int64)]
            L.flexrt_load_state.argtypes = [vp, vp, C.c_int64]
            L.flexrt_get_device_bytes.argtypes = [vp, P(C.c_int64)]
            L.flexrt_get_kernel_times.argtypes = [vp, P(C.c_double), P(C.c_int64), P(C.c_int64)]
            L.flexrt_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
            L.flexrt_last_error.argtypes = [vp]
            L.flexrt_last_error.restype = C.c_char_p
            L.flexrt_destroy.argtypes = [vp]
            L.flexrt_destroy.restype = None
            L.flexrt_default_batch_config.argtypes = [P(BatchConfig)]
            L.flexrt_batch_create.argtypes = [P(BatchConfig), P(vp)]
            L.flexrt_batch_add.argtypes = [vp, P(Grid), P(Box), P(C.c_double), P(Mfp), P(Spectrum), P(Options),
                                           C.c_int32, P(C.c_int32), P(C.c_double), C.c_double, P(C.c_int32)]
            L.flexrt_batch_step.argtypes = [vp]
            L.flexrt_batch_sync.argtypes = [vp]
            L.flexrt_batch_retire.argtypes = [vp, C.c_int32]
            L.flexrt_batch_get_fields.argtypes = [vp, C.c_int32, P(Fields)]
            L.flexrt_batch_get_budget.argtypes = [vp, C.c_int32, P(C.c_double)]
            L.flexrt_batch_get_screen_excess.argtypes = [vp, C.c_int32, P(C.c_double)]
            L.flexrt_batch_get_counts.argtypes = [vp, C.c_int32, P(C.c_int64)]
            L.flexrt_batch_get_segment_counts.argtypes = [vp, C.c_int32, P(C.c_int32)]
            L.flexrt_batch_get_rays.argtypes = [vp, C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int64), P(C.c_int32),
                                                P(C.c_int32), P(C.c_int32), P(C.c_double), P(C.c_int64)]
            L.flexrt_batch_get_rays_merged.argtypes = [vp, C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int32),
                                                       P(C.c_int32), P(C.c_int64), P(C.c_double), P(C.c_int64)]
            L.flexrt_batch_info.argtypes = [vp, P(C.c_int64)]
            L.flexrt_batch_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
            L.flexrt_batch_last_error.argtypes = [vp]
            L.flexrt_batch_last_error.restype = C.c_char_p
            L.flexrt_batch_destroy.argtypes = [vp]
            L.flexrt_batch_destroy.restype = None
            L.flexrt_probe_pixvec.argtypes = [C.c_int32, C.c_int64, C.c_int64, P(C.c_int32)]
            L.flexrt_probe_rotation.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int32, P(C.c_int32)]
            L.flexrt_probe_rates.argtypes = [C.c_int64, P(C.c_float), P(C.c_float)]
            L.flexrt_probe_direction.argtypes = [C.c_int32, C.c_int64, C.c_int64, P(C.c_int32), P(C.c_int32)]
            L.flexrt_probe_traverse.argtypes = [C.c_int64, P(C.c_int64), P(C.c_int32), P(Grid), P(C.c_int32),
                                                P(C.c_float), P(C.c_int32), P(C.c_int32)]
            L.flexrt_probe_traverse_static.argtypes = L.flexrt_probe_traverse.argtypes
            L.flexrt_probe_merge.argtypes = [P(MergeProbe), C.c_int64, P(ProbeRays), C.c_int64, P(ProbeRays),
                                             P(C.c_int64)]
            L.flexrt_probe_merge_pixel.argtypes = [C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int32), C.c_int64,
                                                   P(C.c_int32)]
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _check(status, ctx=None):
    if status != FLEXRT_OK:
        m = lib().flexrt_last_error(ctx)
        raise FlexRTError(status, m.decode() if m else "")


def default_options() -> Options:
    o = Options()
    lib().flexrt_default_options(C.byref(o))
    return o


def _merge_options(o, po):
    o.merge = int(getattr(po, "merge", False))
    o.l_merge = int(getattr(po, "l_merge", 0))
    o.n_ex = float(getattr(po, "n_ex", 16.0))
    o.gamma_iters = int(getattr(po, "gamma_iters", 1))
    o.gen_mode = int(getattr(po, "gen_mode", False))
    o.chi = float(getattr(po, "chi", 0.0))
    o.t_reion = float(getattr(po, "t_reion", 2.0e4))
    o.alpha_pl = float(getattr(po, "alpha_pl", 1.5))


def _merged_fields(getter, out, m):
    """Add the merged-ray fields to a ray dictionary; emitter of a merged ray
    becomes 2^31 + the local index of its merge cell (its rotation key)."""
    n = C.c_int64()
    mg, vx, ds = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.int32)
    P, thr = np.zeros((m, 3), np.int64), np.zeros(m)
    getter(m, _p(mg, C.c_int32), _p(vx, C.c_int32), _p(ds, C.c_int32), _p(P, C.c_int64), _p(thr, C.c_double),
           C.byref(n))
    em = out["emitter"].astype(np.int64)
    out["emitter"] = np.where(mg == 1, (1 << 31) - 1 - em, em)
    out.update(merged=mg.astype(bool), vertex=vx.astype(bool), A=ds, P=P, thr=thr)
    return out


def _problem_structs(prob, keep):
    """C structs (and the arrays they point to, kept alive in `keep`) of a
    problem description."""
    g = Grid(*[int(v) for v in prob.grid])
    b = Box(float(prob.box_cm_comoving), float(prob.redshift))
    sp = prob.spectrum
    fr = np.ascontiguousarray(sp.frac, np.float64)
    sg = np.ascontiguousarray(sp.sigma_cm2, np.float64)
    eh = np.ascontiguousarray(sp.eheat_erg, np.float64)
    keep += [fr, sg, eh]
    s = Spectrum(int(sp.nbins), _p(fr, C.c_double), _p(sg, C.c_double), _p(eh, C.c_double))
    m = prob.mfp
    mf = Mfp(int(m.mode), m.lambda0_cm_comoving, m.delta_exp, m.gamma_ref, m.gamma_exp, m.gamma_floor,
             m.xion_threshold, m.nH_mean)
    o = default_options()
    po = prob.options
    o.l_src, o.l_max = po.l_src, po.l_max
    o.n_ray_min, o.eps_term = po.n_ray_min, po.eps_term
    o.seed = po.seed
    o.rotate, o.isothermal, o.rates, o.chem_iters = int(po.rotate), int(po.isothermal), int(po.rates), po.chem_iters
    o.alpha_B_const, o.x_init, o.T_init = po.alpha_B_const, po.x_init, po.T_init
    _merge_options(o, po)
    return g, b, s, mf, o


class Batch:
    """Many simulations advanced together (flexrt_batch_*): members are added
    and retired between steps; one step advances every active member."""

    def __init__(self, max_sims=64, max_grid=160, nbins=3, ray_capacity=0, cell_capacity=None,
                 emitter_capacity=65536, use_graph=True, keep_diagnostics=False, n_ray_min=3.0, stream=None,
                 merge_l_max=-1, gen_capable=False):
        L = lib()
        c = BatchConfig()
        L.flexrt_default_batch_config(C.byref(c))
        c.merge_l_max = int(merge_l_max)
        c.gen_capable = int(gen_capable)
        c.max_sims, c.max_grid, c.nbins, c.n_ray_min = max_sims, max_grid, nbins, n_ray_min
        c.ray_capacity = int(ray_capacity)
        c.cell_capacity = int(cell_capacity if cell_capacity is not None else max_sims * max_grid ** 3)
        c.emitter_capacity = int(emitter_capacity)
        c.use_graph, c.keep_diagnostics = int(use_graph), int(keep_diagnostics)
        c.cuda_stream = stream
        h = C.c_void_p()
        st = L.flexrt_batch_create(C.byref(c), C.byref(h))
        if st != FLEXRT_OK:
            m = L.flexrt_last_error(None)
            raise FlexRTError(st, m.decode() if m else "")
        self._h = h
        self.members = {}

    def _check(self, st):
        if st != FLEXRT_OK:
            m = lib().flexrt_batch_last_error(self._h)
            raise FlexRTError(st, m.decode() if m else "")

    def add(self, prob) -> int:
        keep = []
        g, b, s, mf, o = _problem_structs(prob, keep)
        nH = np.ascontiguousarray(prob.nH, np.float64).reshape(-1)
        cells = np.ascontiguousarray(np.asarray(prob.source_cells, np.int32).reshape(-1, 3))
        nd = np.ascontiguousarray(np.asarray(prob.source_ndot, np.float64).reshape(-1))
        slot = C.c_int32()
        self._check(lib().flexrt_batch_add(self._h, C.byref(g), C.byref(b), _p(nH, C.c_double), C.byref(mf),
                                           C.byref(s), C.byref(o), len(nd), _p(cells, C.c_int32),
                                           _p(nd, C.c_double), float(prob.dt), C.byref(slot)))
        self.members[slot.value] = (nH.size, int(prob.spectrum.nbins))
        return slot.value

    def step(self):
        self._check(lib().flexrt_batch_step(self._h))

    def sync(self):
        self._check(lib().flexrt_batch_sync(self._h))

    def retire(self, slot):
        self._check(lib().flexrt_batch_retire(self._h, int(slot)))
        self.members.pop(slot, None)

    def fields(self, slot, which=("gamma_HI", "x_HII", "T", "n_HI")):
        n = self.members[slot][0]
        out = {k: np.zeros(n) for k in which}
        f = Fields(*[(_p(out[k], C.c_double) if k in out else None) for k in ("gamma_HI", "x_HII", "T", "n_HI")])
        self._check(lib().flexrt_batch_get_fields(self._h, int(slot), C.byref(f)))
        return out

    def budget(self, slot):
        b = np.zeros(4)
        self._check(lib().flexrt_batch_get_budget(self._h, int(slot), _p(b, C.c_double)))
        return b

    def screen_excess(self, slot):
        v = np.zeros(1)
        self._check(lib().flexrt_batch_get_screen_excess(self._h, int(slot), _p(v, C.c_double)))
        return float(v[0])

    def counts(self, slot):
        c = np.zeros(6, np.int64)
        self._check(lib().flexrt_batch_get_counts(self._h, int(slot), _p(c, C.c_int64)))
        return dict(rays=int(c[0]), segments_last=int(c[1]), segments_total=int(c[2]), step=int(c[3]),
                    capacity=int(c[4]), rays_marched_last=int(c[5]))

    def segment_counts(self, slot):
        s = np.zeros(self.members[slot][0], np.int32)
        self._check(lib().flexrt_batch_get_segment_counts(self._h, int(slot), _p(s, C.c_int32)))
        return s

    def rays(self, slot):
        nb = self.members[slot][1]
        n = C.c_int64()
        self._check(lib().flexrt_batch_get_rays(self._h, int(slot), 0, None, None, None, None, None, None,
                                                C.byref(n)))
        m = n.value
        lv, pix = np.zeros(m, np.int32), np.zeros(m, np.int64)
        em, bi = np.zeros(m, np.int32), np.zeros(m, np.int32)
        d, N = np.zeros((m, 3), np.int32), np.zeros((m, nb))
        self._check(lib().flexrt_batch_get_rays(self._h, int(slot), m, _p(lv, C.c_int32), _p(pix, C.c_int64),
                                                _p(em, C.c_int32), _p(bi, C.c_int32), _p(d, C.c_int32),
                                                _p(N, C.c_double), C.byref(n)))
        out = dict(level=lv, pixel=pix, emitter=em, birth=bi, dir=d, N=N)
        return _merged_fields(lambda *a: self._check(lib().flexrt_batch_get_rays_merged(self._h, int(slot), *a)),
                              out, m)

    def ionized_volume(self, slot):
        x = np.zeros(self.members[slot][0])
        self._check(lib().flexrt_batch_get_ionized_volume(self._h, int(slot), _p(x, C.c_double)))
        return x

    def info(self):
        o = np.zeros(6, np.int64)
        self._check(lib().flexrt_batch_info(self._h, _p(o, C.c_int64)))
        return dict(active=int(o[0]), cells_free=int(o[1]), emitters_free=int(o[2]), ray_capacity=int(o[3]),
                    queue_used=int(o[4]), slots_free=int(o[5]))

    def set_launch(self, agg, minb, blocks_per_sm=0, threads=0, slab=0):
        self._check(lib().flexrt_batch_set_launch(self._h, int(agg), int(minb), int(blocks_per_sm), int(threads),
                                                  int(slab)))

    def close(self):
        if getattr(self, "_h", None):
            lib().flexrt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """One simulation on the GPU, created from a problem description with the
    attributes grid, box_cm_comoving, redshift, nH, spectrum (nbins, frac,
    sigma_cm2, eheat_erg), mfp, options, source_cells, source_ndot."""

    def __init__(self, prob, ray_capacity: int = 0, keep_diagnostics: bool = False, stream=None,
                 device_bytes_max: int = 0):
        L = lib()
        g = Grid(*[int(v) for v in prob.grid])
        b = Box(float(prob.box_cm_comoving), float(prob.redshift))
        sp = prob.spectrum
        self._frac = np.ascontiguousarray(sp.frac, np.float64)
        self._sig = np.ascontiguousarray(sp.sigma_cm2, np.float64)
        self._eh = np.ascontiguousarray(sp.eheat_erg, np.float64)
        s = Spectrum(int(sp.nbins), _p(self._frac, C.c_double), _p(self._sig, C.c_double), _p(self._eh, C.c_double))
        m = prob.mfp
        mf = Mfp(int(m.mode), m.lambda0_cm_comoving, m.delta_exp, m.gamma_ref, m.gamma_exp, m.gamma_floor,
                 m.xion_threshold, m.nH_mean)
        o = default_options()
        po = prob.options
        o.l_src, o.l_max = po.l_src, po.l_max
        o.n_ray_min, o.eps_term = po.n_ray_min, po.eps_term
        o.seed = po.seed
        o.rotate, o.isothermal, o.rates, o.chem_iters = int(po.rotate), int(po.isothermal), int(po.rates), po.chem_iters
        o.alpha_B_const, o.x_init, o.T_init = po.alpha_B_const, po.x_init, po.T_init
        _merge_options(o, po)
        o.ray_capacity = int(ray_capacity)
        o.keep_diagnostics = int(keep_diagnostics)
        o.cuda_stream = stream
        o.device_bytes_max = int(device_bytes_max)
        nH = np.ascontiguousarray(prob.nH, np.float64).reshape(-1)
        self.ncell = nH.size
        self.nb = int(sp.nbins)
        h = C.c_void_p()
        st = L.flexrt_create(C.byref(g), C.byref(b), _p(nH, C.c_double), C.byref(mf), C.byref(s), C.byref(o),
                             C.byref(h))
        if st != FLEXRT_OK:
            raise FlexRTError(st, "flexrt_create failed: " + (L.flexrt_last_error(None) or b"").decode())
        self._h = h
        if len(prob.source_ndot):
            self.add_sources(prob.source_cells, prob.source_ndot)

    def add_sources(self, cells, ndot):
        cells = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1, 3))
        ndot = np.ascontiguousarray(np.asarray(ndot, np.float64).reshape(-1))
        _check(lib().flexrt_add_sources(self._h, len(ndot), _p(cells, C.c_int32), _p(ndot, C.c_double)), self._h)

    def step(self, dt: float):
        _check(lib().flexrt_step(self._h, float(dt)), self._h)

    def step_stage(self, dt: float, stage: int):
        """One step in two stages (1: emission and marches; 2: merge,
        chemistry, commit); rays() in between returns the march's output."""
        _check(lib().flexrt_step_stage(self._h, float(dt), int(stage)), self._h)

    def sync(self):
        _check(lib().flexrt_sync(self._h), self._h)

    def reset(self):
        _check(lib().flexrt_reset(self._h), self._h)

    def fields(self, which=("gamma_HI", "x_HII", "T", "n_HI")):
        out = {k: np.zeros(self.ncell) for k in which}
        f = Fields(*[(_p(out[k], C.c_double) if k in out else None) for k in ("gamma_HI", "x_HII", "T", "n_HI")])
        _check(lib().flexrt_get_fields(self._h, C.byref(f)), self._h)
        return out

    def budget(self):
        b = np.zeros(4)
        _check(lib().flexrt_get_budget(self._h, _p(b, C.c_double)), self._h)
        return b

    def screen_excess(self):
        """Photons the moving screens absorbed beyond their atoms (Generalized
        mode; part of the absorbed photons that ionised nothing)."""
        v = np.zeros(1)
        _check(lib().flexrt_get_screen_excess(self._h, _p(v, C.c_double)), self._h)
        return float(v[0])

    def counts(self):
        c = np.zeros(6, np.int64)
        _check(lib().flexrt_get_counts(self._h, _p(c, C.c_int64)), self._h)
        return dict(rays=int(c[0]), segments_last=int(c[1]), segments_total=int(c[2]), step=int(c[3]),
                    capacity=int(c[4]), rays_marched_last=int(c[5]))

    def segment_counts(self):
        s = np.zeros(self.ncell, np.int32)
        _check(lib().flexrt_get_segment_counts(self._h, _p(s, C.c_int32)), self._h)
        return s

    def rays(self, cap=None):
        n = C.c_int64()
        _check(lib().flexrt_get_rays(self._h, 0, None, None, None, None, None, None, C.byref(n)), self._h)
        m = n.value if cap is None else min(cap, n.value)
        lv = np.zeros(m, np.int32)
        pix = np.zeros(m, np.int64)
        em = np.zeros(m, np.int32)
        bi = np.zeros(m, np.int32)
        d = np.zeros((m, 3), np.int32)
        N = np.zeros((m, self.nb))
        _check(lib().flexrt_get_rays(self._h, m, _p(lv, C.c_int32), _p(pix, C.c_int64), _p(em, C.c_int32),
                                     _p(bi, C.c_int32), _p(d, C.c_int32), _p(N, C.c_double), C.byref(n)), self._h)
        out = dict(level=lv, pixel=pix, emitter=em, birth=bi, dir=d, N=N)
        return _merged_fields(lambda *a: _check(lib().flexrt_get_rays_merged(self._h, *a), self._h), out, m)

    def save_state(self) -> np.ndarray:
        """Checkpoint of the simulation as a host byte array."""
        n = C.c_int64()
        _check(lib().flexrt_save_state(self._h, None, 0, C.byref(n)), self._h)
        buf = np.zeros(n.value, np.uint8)
        _check(lib().flexrt_save_state(self._h, buf.ctypes.data_as(C.c_void_p), n.value, C.byref(n)), self._h)
        return buf

    def load_state(self, buf):
        """Restore a checkpoint made by save_state of the same simulation."""
        buf = np.ascontiguousarray(np.asarray(buf, np.uint8))
        _check(lib().flexrt_load_state(self._h, buf.ctypes.data_as(C.c_void_p), buf.size), self._h)

    def device_bytes(self) -> int:
        n = C.c_int64()
        _check(lib().flexrt_get_device_bytes(self._h, C.byref(n)), self._h)
        return int(n.value)

    def ionized_volume(self):
        """Generalized mode: the highly ionised volume fraction per cell."""
        x = np.zeros(self.ncell)
        _check(lib().flexrt_get_ionized_volume(self._h, _p(x, C.c_double)), self._h)
        return x

    def profile(self, enable=True):
        _check(lib().flexrt_profile(self._h, int(enable)), self._h)

    def kernel_times(self):
        ms = np.zeros(4)
        ln = np.zeros(4, np.int64)
        rays = np.zeros(1, np.int64)
        _check(lib().flexrt_get_kernel_times(self._h, _p(ms, C.c_double), _p(ln, C.c_int64), _p(rays, C.c_int64)),
               self._h)
        names = ("emit", "march", "chem", "merge")
        return dict(zip(names, ms)), dict(zip(names, ln)), int(rays[0])

    def set_launch(self, agg: int, minb: int, blocks_per_sm: int = 0, threads: int = 0, slab: int = 0):
        _check(lib().flexrt_set_launch(self._h, int(agg), int(minb), int(blocks_per_sm), int(threads), int(slab)),
               self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().flexrt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------------------
# device-function probes
# -------------------------------------------------------------------------
def probe_pixvec(level: int, p0: int, n: int) -> np.ndarray:
    out = np.zeros((n, 3), np.int32)
    _check(lib().flexrt_probe_pixvec(level, p0, n, _p(out, C.c_int32)))
    return out


def probe_rates(T) -> np.ndarray:
    """The chemistry kernel's rate fits at temperatures T: columns alpha_B,
    alpha_A, C_HI and the cooling rate (unit densities, no Compton term)."""
    T = np.ascontiguousarray(np.asarray(T, np.float32).ravel())
    out = np.zeros((len(T), 4), np.float32)
    _check(lib().flexrt_probe_rates(len(T), _p(T, C.c_float), _p(out, C.c_float)))
    return out


def probe_rotation(seed: int, emitter: int, step: int, rotate: bool = True) -> np.ndarray:
    out = np.zeros(9, np.int32)
    _check(lib().flexrt_probe_rotation(seed, emitter, step, int(rotate), _p(out, C.c_int32)))
    return out.reshape(3, 3)


def probe_direction(level: int, p0: int, n: int, Rq) -> np.ndarray:
    Rq = np.ascontiguousarray(np.asarray(Rq, np.int32).reshape(9))
    out = np.zeros((n, 3), np.int32)
    _check(lib().flexrt_probe_direction(level, p0, n, _p(Rq, C.c_int32), _p(out, C.c_int32)))
    return out


STATIC_MAX_RAYS = 32768


def probe_merge_pixel(level: int, d, Rq) -> np.ndarray:
    """Merge-sphere pixels (Sec. 3.3) of fixed-point directions d [n,3] on the
    sphere rotated by Rq (3x3 int32, or [n,3,3]: one sphere per direction),
    decided on the GPU."""
    d = np.ascontiguousarray(np.asarray(d, np.int32).reshape(-1, 3))
    Rq = np.asarray(Rq, np.int32)
    nrot = 1 if Rq.size == 9 else len(d)
    Rq = np.ascontiguousarray(Rq.reshape(nrot * 9))
    out = np.zeros(len(d), np.int32)
    _check(lib().flexrt_probe_merge_pixel(int(level), len(d), _p(d, C.c_int32), _p(Rq, C.c_int32), nrot,
                                          _p(out, C.c_int32)))
    return out


def probe_merge(grid, nbins, l_src, l_max, l_merge, k_ex, seed, rotate, step, eps_term, emitter_cells,
                emitter_n0, rays):
    """Run the merge step's kernels (Sec. 3.3) on the rays `rays` of one
    simulation as they stand after the march of `step`.  `rays`: level,
    pixel, emitter (2^31 + local cell for a merged ray), birth, dir [n,3],
    N [n,nbins] (code photons, float32), and for merged rays merged, vertex,
    A, P [n,3], thr (code photons).  Returns the rays after the merge in the
    same form."""
    n = len(rays["level"])
    merged = np.asarray(rays.get("merged", np.zeros(n, bool)), bool)
    u32 = lambda x: np.ascontiguousarray(np.asarray(x).astype(np.int64).astype(np.uint32))
    i32 = lambda x: np.ascontiguousarray(np.asarray(x).astype(np.int32))
    pl = u32((np.asarray(rays["level"], np.int64) << 28) | np.asarray(rays["pixel"], np.int64))
    em64 = np.asarray(rays["emitter"]).astype(np.int64)
    em = u32(np.where(merged, (1 << 31) | (em64 - (1 << 31)), em64))
    bi = i32(rays["birth"])
    d = i32(np.asarray(rays["dir"]).reshape(n, 3))
    ph = np.ascontiguousarray(np.asarray(rays["N"], np.float32).reshape(n, nbins))
    pos = i32(np.where(merged[:, None], np.asarray(rays.get("P", np.zeros((n, 3)))), 0).reshape(n, 3))
    aux = u32(np.where(merged, (np.asarray(rays.get("vertex", np.zeros(n)), np.int64) << 31)
                       | np.asarray(rays.get("A", np.zeros(n)), np.int64), 0))
    thr = np.ascontiguousarray(np.where(merged, np.asarray(rays.get("thr", np.zeros(n))), 0).astype(np.float32))
    keep = [pl, em, bi, d, ph, pos, aux, thr]
    rin = ProbeRays(*[_p(x, t) for x, t in zip(keep, (C.c_uint32, C.c_uint32, C.c_int32, C.c_int32, C.c_float,
                                                      C.c_int32, C.c_uint32, C.c_float))])
    cap = max(n, 1)
    o = dict(pixlev=np.zeros(cap, np.uint32), emitter=np.zeros(cap, np.uint32), birth=np.zeros(cap, np.int32),
             dir=np.zeros((cap, 3), np.int32), N=np.zeros((cap, nbins), np.float32), P=np.zeros((cap, 3), np.int32),
             aux=np.zeros(cap, np.uint32), thr=np.zeros(cap, np.float32))
    rout = ProbeRays(*[_p(o[k], t) for k, t in zip(("pixlev", "emitter", "birth", "dir", "N", "P", "aux", "thr"),
                                                    (C.c_uint32, C.c_uint32, C.c_int32, C.c_int32, C.c_float,
                                                     C.c_int32, C.c_uint32, C.c_float))])
    ec = np.ascontiguousarray(np.asarray(emitter_cells, np.int32).reshape(-1, 3))
    n0 = np.ascontiguousarray(np.asarray(emitter_n0, np.float32).reshape(-1))
    mp = MergeProbe(int(grid[0]), int(grid[1]), int(grid[2]), int(nbins), int(l_src), int(l_max), int(l_merge),
                    int(k_ex), int(seed), int(rotate), int(step), float(eps_term), len(n0), _p(ec, C.c_int32),
                    _p(n0, C.c_float))
    nout = C.c_int64()
    _check(lib().flexrt_probe_merge(C.byref(mp), n, C.byref(rin), cap, C.byref(rout), C.byref(nout)))
    m = nout.value
    em_o = o["emitter"][:m].astype(np.int64)
    mg = (em_o & (1 << 31)) != 0
    return dict(level=(o["pixlev"][:m] >> 28).astype(np.int32), pixel=(o["pixlev"][:m] & 0x0FFFFFFF).astype(np.int64),
                emitter=em_o, birth=o["birth"][:m], dir=o["dir"][:m], N=o["N"][:m].astype(np.float64),
                merged=mg, vertex=mg & ((o["aux"][:m] >> 31) == 1), A=np.where(mg, o["aux"][:m] & 0xffff, 0),
                P=np.where(mg[:, None], o["P"][:m].astype(np.int64), 0),
                thr=np.where(mg, o["thr"][:m].astype(np.float64), 0.0))


def probe_traverse_static(p0, d, grid):
    """probe_traverse through the entry point that allocates no device
    memory (at most STATIC_MAX_RAYS rays per call)."""
    return probe_traverse(p0, d, grid, _entry="flexrt_probe_traverse_static")


def probe_traverse(p0, d, grid, _entry="flexrt_probe_traverse"):
    p0 = np.ascontiguousarray(np.asarray(p0, np.int64).reshape(-1, 3))
    d = np.ascontiguousarray(np.asarray(d, np.int32).reshape(-1, 3))
    n = len(p0)
    cells = np.zeros((n, 4, 3), np.int32)
    ds = np.zeros((n, 4), np.float32)
    nseg = np.zeros(n, np.int32)
    esc = np.zeros(n, np.int32)
    g = Grid(*[int(v) for v in grid])
    fn = getattr(lib(), _entry)
    _check(fn(n, _p(p0, C.c_int64), _p(d, C.c_int32), C.byref(g), _p(cells, C.c_int32),
              _p(ds, C.c_float), _p(nseg, C.c_int32), _p(esc, C.c_int32)))
    return cells, ds, nseg, esc.astype(bool)
