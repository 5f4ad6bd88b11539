// flexrt_api.cu -- the C ABI declared in include/flexrt.h.
//
// A flexrt_ctx is an engine with one simulation slot, stepped by direct
// launches; a flexrt_batch is an engine with many slots whose step (one RT
// step of every active simulation) is replayed from a CUDA graph.  Both run
// the same kernels; every size the kernels need is read from device memory.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "../../include/flexrt.h"
#include "frt_engine.h"

using namespace frt;

namespace frt {
static thread_local std::string g_free_err;
void set_free_error(const std::string &msg) { g_free_err = msg; }
}  // namespace frt

struct flexrt_ctx {
    Engine eng;
    int slot = 0;
};

struct flexrt_batch {
    Engine eng;
};

extern "C" void flexrt_default_options(flexrt_options *o) {
    std::memset(o, 0, sizeof(*o));
    o->l_src = 0;
    o->l_max = FLEXRT_MAX_LEVEL;
    o->n_ray_min = 3.0;
    o->eps_term = 1e-10;
    o->seed = 1;
    o->rotate = 1;
    o->isothermal = 1;
    o->rates = 0;
    o->chem_iters = 5;
    o->alpha_B_const = 2.59e-13;
    o->x_init = 1.2e-3;
    o->T_init = 1e4;
}

static flexrt_status free_fail(flexrt_status s, const std::string &m) {
    frt::set_free_error(m);
    return s;
}

extern "C" flexrt_status flexrt_create(const flexrt_grid *grid, const flexrt_box *box, const double *n_H,
                                       const flexrt_mfp *mfp, const flexrt_spectrum *sp,
                                       const flexrt_options *opt_in, flexrt_ctx **out) {
    if (!out) return FLEXRT_E_INVALID;
    *out = nullptr;
    flexrt_options opt;
    if (opt_in) opt = *opt_in; else flexrt_default_options(&opt);
    SimDev h;
    std::string err;
    flexrt_status s = Engine::make_sim(grid, box, n_H, mfp, sp, &opt, h, err);
    if (s != FLEXRT_OK) return free_fail(s, "flexrt_create: " + err);
    flexrt_ctx *c = new (std::nothrow) flexrt_ctx();
    if (!c) return FLEXRT_E_OOM;
    EngineConfig cfg;
    cfg.nb = sp->nbins;
    cfg.max_sims = 1;
    cfg.ray_capacity = opt.ray_capacity;
    cfg.cell_capacity = h.ncell;
    cfg.emitter_capacity = 0;
    cfg.max_grid = std::max(grid->nx, std::max(grid->ny, grid->nz));
    cfg.l_max = opt.l_max;
    cfg.n_ray_min = opt.n_ray_min;
    cfg.keep_diagnostics = opt.keep_diagnostics != 0;
    cfg.use_graph = false;
    cfg.stream = opt.cuda_stream;
    s = c->eng.init(cfg);
    if (s == FLEXRT_OK) s = c->eng.add_sim(h, n_H, &c->slot);
    if (s != FLEXRT_OK) {
        free_fail(s, "flexrt_create: " + c->eng.error());
        delete c;
        return s;
    }
    *out = c;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_add_sources(flexrt_ctx *c, int32_t n, const int32_t *ijk, const double *ndot) {
    if (!c) return FLEXRT_E_INVALID;
    return c->eng.add_sources(c->slot, n, ijk, ndot);
}

extern "C" flexrt_status flexrt_step(flexrt_ctx *c, double dt) {
    if (!c) return FLEXRT_E_INVALID;
    flexrt_status s = c->eng.set_dt(c->slot, dt);
    if (s != FLEXRT_OK) return s;
    return c->eng.step();
}

extern "C" flexrt_status flexrt_sync(flexrt_ctx *c) { return c ? c->eng.sync() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_reset(flexrt_ctx *c) { return c ? c->eng.reset_all() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_get_fields(flexrt_ctx *c, flexrt_fields *f) {
    return c ? c->eng.fields(c->slot, f) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_budget(flexrt_ctx *c, double out[4]) {
    return c ? c->eng.budget(c->slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_counts(flexrt_ctx *c, int64_t out[6]) {
    return c ? c->eng.counts(c->slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_segment_counts(flexrt_ctx *c, int32_t *out) {
    return c ? c->eng.segment_counts(c->slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_rays(flexrt_ctx *c, int64_t cap, int32_t *level, int64_t *pixel,
                                         int32_t *emitter, int32_t *birth, int32_t *dir, double *photons,
                                         int64_t *n) {
    return c ? c->eng.rays(c->slot, cap, level, pixel, emitter, birth, dir, photons, n) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_profile(flexrt_ctx *c, int32_t enable) {
    return c ? c->eng.profile(enable != 0) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_kernel_times(flexrt_ctx *c, double ms[3], int64_t launches[3],
                                                 int64_t march_rays[1]) {
    if (!c || !ms || !launches) return FLEXRT_E_INVALID;
    return c->eng.kernel_times(ms, launches, march_rays);
}
extern "C" flexrt_status flexrt_set_launch(flexrt_ctx *c, int32_t agg, int32_t minb, int32_t blocks_per_sm) {
    return c ? c->eng.set_launch(agg, minb, blocks_per_sm) : FLEXRT_E_INVALID;
}
extern "C" const char *flexrt_last_error(const flexrt_ctx *c) {
    return c ? c->eng.error().c_str() : frt::g_free_err.c_str();
}
extern "C" void flexrt_destroy(flexrt_ctx *c) { delete c; }

// ---------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------
extern "C" void flexrt_default_batch_config(flexrt_batch_config *b) {
    std::memset(b, 0, sizeof(*b));
    b->max_sims = 64;
    b->max_grid = 160;
    b->nbins = 3;
    b->n_ray_min = 3.0;
    b->use_graph = 1;
}

extern "C" flexrt_status flexrt_batch_create(const flexrt_batch_config *bc, flexrt_batch **out) {
    if (!out || !bc) return FLEXRT_E_INVALID;
    *out = nullptr;
    if (bc->max_sims < 1 || bc->max_sims > 512 || bc->max_grid < 1 || bc->max_grid > 1000 || bc->nbins < 1 ||
        bc->nbins > FLEXRT_MAX_BINS || bc->cell_capacity < 1 || bc->emitter_capacity < 1)
        return free_fail(FLEXRT_E_INVALID, "flexrt_batch_create: bad configuration");
    flexrt_batch *b = new (std::nothrow) flexrt_batch();
    if (!b) return FLEXRT_E_OOM;
    EngineConfig cfg;
    cfg.nb = bc->nbins;
    cfg.max_sims = bc->max_sims;
    cfg.ray_capacity = bc->ray_capacity;
    cfg.cell_capacity = bc->cell_capacity;
    cfg.emitter_capacity = bc->emitter_capacity;
    cfg.max_grid = bc->max_grid;
    cfg.l_max = FLEXRT_MAX_LEVEL;
    cfg.n_ray_min = bc->n_ray_min > 0 ? bc->n_ray_min : 3.0;
    cfg.keep_diagnostics = bc->keep_diagnostics != 0;
    cfg.use_graph = bc->use_graph != 0;
    cfg.stream = bc->cuda_stream;
    flexrt_status s = b->eng.init(cfg);
    if (s != FLEXRT_OK) {
        free_fail(s, "flexrt_batch_create: " + b->eng.error());
        delete b;
        return s;
    }
    *out = b;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_batch_add(flexrt_batch *b, const flexrt_grid *grid, const flexrt_box *box,
                                          const double *n_H, const flexrt_mfp *mfp, const flexrt_spectrum *sp,
                                          const flexrt_options *opt, int32_t n_sources, const int32_t *cell_ijk,
                                          const double *ndot, double dt_s, int32_t *slot) {
    if (!b || !slot) return FLEXRT_E_INVALID;
    if (!(dt_s > 0)) return b->eng.fail(FLEXRT_E_INVALID, "dt must be positive");
    SimDev h;
    std::string err;
    flexrt_status s = Engine::make_sim(grid, box, n_H, mfp, sp, opt, h, err);
    if (s != FLEXRT_OK) return b->eng.fail(s, err);
    int sl = -1;
    s = b->eng.add_sim(h, n_H, &sl);
    if (s != FLEXRT_OK) return s;
    s = b->eng.add_sources(sl, n_sources, cell_ijk, ndot);
    if (s == FLEXRT_OK) s = b->eng.set_dt(sl, dt_s);
    if (s != FLEXRT_OK) {
        b->eng.retire(sl);
        return s;
    }
    *slot = sl;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_batch_step(flexrt_batch *b) { return b ? b->eng.step() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_batch_sync(flexrt_batch *b) { return b ? b->eng.sync() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_batch_retire(flexrt_batch *b, int32_t slot) {
    return b ? b->eng.retire(slot) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_fields(flexrt_batch *b, int32_t slot, flexrt_fields *f) {
    return b ? b->eng.fields(slot, f) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_budget(flexrt_batch *b, int32_t slot, double out[4]) {
    return b ? b->eng.budget(slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_counts(flexrt_batch *b, int32_t slot, int64_t out[6]) {
    return b ? b->eng.counts(slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_rays(flexrt_batch *b, int32_t slot, int64_t cap, int32_t *level,
                                               int64_t *pixel, int32_t *emitter, int32_t *birth, int32_t *dir,
                                               double *photons, int64_t *n) {
    return b ? b->eng.rays(slot, cap, level, pixel, emitter, birth, dir, photons, n) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_info(flexrt_batch *b, int64_t out[6]) {
    if (!b || !out) return FLEXRT_E_INVALID;
    long long q = 0;
    flexrt_status s = b->eng.queue_used(&q);
    if (s != FLEXRT_OK) return s;
    out[0] = b->eng.active_count();
    out[1] = b->eng.cells_free();
    out[2] = b->eng.emitters_free();
    out[3] = b->eng.ray_capacity();
    out[4] = q;
    out[5] = b->eng.free_slots();
    return FLEXRT_OK;
}
extern "C" flexrt_status flexrt_batch_set_launch(flexrt_batch *b, int32_t agg, int32_t minb, int32_t bps) {
    return b ? b->eng.set_launch(agg, minb, bps) : FLEXRT_E_INVALID;
}
extern "C" const char *flexrt_batch_last_error(const flexrt_batch *b) {
    return b ? b->eng.error().c_str() : frt::g_free_err.c_str();
}
extern "C" void flexrt_batch_destroy(flexrt_batch *b) { delete b; }

// ---------------------------------------------------------------------------
// probes
// ---------------------------------------------------------------------------
namespace {
template <typename T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)); }
};
}  // namespace

extern "C" flexrt_status flexrt_probe_pixvec(int32_t level, int64_t p0, int64_t n, int32_t *out) {
    if (level < 0 || level > FLEXRT_MAX_LEVEL || n < 0 || p0 < 0 || p0 + n > (12LL << (2 * level)) || (n && !out))
        return FLEXRT_E_INVALID;
    DevBuf<int32_t> d;
    if (d.alloc(3 * n) != cudaSuccess) return FLEXRT_E_OOM;
    if (launch_probe_pixvec(level, p0, n, d.p, 0) != cudaSuccess) return FLEXRT_E_CUDA;
    if (cudaMemcpy(out, d.p, 3 * n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return FLEXRT_E_CUDA;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_probe_rotation(uint64_t seed, int64_t e, int64_t s, int32_t rotate, int32_t *out) {
    if (!out) return FLEXRT_E_INVALID;
    DevBuf<int32_t> d;
    if (d.alloc(9) != cudaSuccess) return FLEXRT_E_OOM;
    if (launch_probe_rotation(seed, e, s, rotate, d.p, 0) != cudaSuccess) return FLEXRT_E_CUDA;
    if (cudaMemcpy(out, d.p, 9 * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return FLEXRT_E_CUDA;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_probe_direction(int32_t level, int64_t p0, int64_t n, const int32_t *Rq,
                                                int32_t *out) {
    if (level < 0 || level > FLEXRT_MAX_LEVEL || n < 0 || p0 < 0 || p0 + n > (12LL << (2 * level)) || !Rq ||
        (n && !out))
        return FLEXRT_E_INVALID;
    int dev = 0;
    cudaGetDevice(&dev);
    const int4 *tab = nullptr;
    int lt = std::min(level, 8);
    if (get_pixtab(dev, lt, 0, &tab) != cudaSuccess) return FLEXRT_E_CUDA;
    DevBuf<int32_t> dr, d;
    if (dr.alloc(9) != cudaSuccess || d.alloc(3 * n) != cudaSuccess) return FLEXRT_E_OOM;
    if (cudaMemcpy(dr.p, Rq, 9 * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) return FLEXRT_E_CUDA;
    if (launch_probe_direction(level, p0, n, dr.p, tab, lt, d.p, 0) != cudaSuccess) return FLEXRT_E_CUDA;
    if (cudaMemcpy(out, d.p, 3 * n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return FLEXRT_E_CUDA;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_probe_traverse(int64_t n, const int64_t *p0, const int32_t *dir,
                                               const flexrt_grid *g, int32_t *cells, float *ds, int32_t *nseg,
                                               int32_t *escaped) {
    if (n < 0 || !g || (n && (!p0 || !dir || !cells || !ds || !nseg || !escaped))) return FLEXRT_E_INVALID;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (dir[i] > (1 << 21) || dir[i] < -(1 << 21)) return FLEXRT_E_INVALID;
    DevBuf<long long> dp;
    DevBuf<int32_t> dd, dc, dn, de;
    DevBuf<float> dsb;
    if (dp.alloc(3 * n) != cudaSuccess || dd.alloc(3 * n) != cudaSuccess || dc.alloc(12 * n) != cudaSuccess ||
        dn.alloc(n) != cudaSuccess || de.alloc(n) != cudaSuccess || dsb.alloc(4 * n) != cudaSuccess)
        return FLEXRT_E_OOM;
    if (cudaMemcpy(dp.p, p0, 3 * n * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dd.p, dir, 3 * n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dc.p, 0xff, 12 * n * sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(dsb.p, 0, 4 * n * sizeof(float)) != cudaSuccess)
        return FLEXRT_E_CUDA;
    if (launch_probe_traverse(n, dp.p, dd.p, g->nx, g->ny, g->nz, dc.p, dsb.p, dn.p, de.p, 0) != cudaSuccess)
        return FLEXRT_E_CUDA;
    if (cudaMemcpy(cells, dc.p, 12 * n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ds, dsb.p, 4 * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nseg, dn.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(escaped, de.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FLEXRT_E_CUDA;
    return FLEXRT_OK;
}
