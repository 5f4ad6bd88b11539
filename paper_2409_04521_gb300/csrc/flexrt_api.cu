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
    o->merge = 0;
    o->l_merge = 0;
    o->n_ex = 16.0;
    o->gamma_iters = 1;
    o->gen_mode = 0;
    o->chi = 0.0;
    o->t_reion = 2.0e4;
    o->alpha_pl = 1.5;
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
    cfg.merge_l_max = opt.merge ? opt.l_merge : -1;
    cfg.gen_capable = opt.gen_mode != 0;
    cfg.device_bytes_max = opt.device_bytes_max;
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

extern "C" flexrt_status flexrt_step_stage(flexrt_ctx *c, double dt, int32_t stage) {
    if (!c) return FLEXRT_E_INVALID;
    if (stage == 1) {
        flexrt_status s = c->eng.set_dt(c->slot, dt);
        if (s != FLEXRT_OK) return s;
    }
    return c->eng.step_stage(stage);
}

extern "C" flexrt_status flexrt_sync(flexrt_ctx *c) { return c ? c->eng.sync() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_reset(flexrt_ctx *c) { return c ? c->eng.reset_all() : FLEXRT_E_INVALID; }
extern "C" flexrt_status flexrt_get_fields(flexrt_ctx *c, flexrt_fields *f) {
    return c ? c->eng.fields(c->slot, f) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_budget(flexrt_ctx *c, double out[4]) {
    return c ? c->eng.budget(c->slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_screen_excess(flexrt_ctx *c, double *photons) {
    return c ? c->eng.screen_excess(c->slot, photons) : FLEXRT_E_INVALID;
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
extern "C" flexrt_status flexrt_get_ionized_volume(flexrt_ctx *c, double *x_ion) {
    return c ? c->eng.ionized_volume(c->slot, x_ion) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_rays_merged(flexrt_ctx *c, int64_t cap, int32_t *merged, int32_t *vertex,
                                                int32_t *dist, int64_t *pos, double *thr, int64_t *n) {
    return c ? c->eng.rays_merged(c->slot, cap, merged, vertex, dist, pos, thr, n) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_save_state(flexrt_ctx *c, void *buf, int64_t cap, int64_t *bytes) {
    return c ? c->eng.save_state(c->slot, buf, cap, bytes) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_load_state(flexrt_ctx *c, const void *buf, int64_t bytes) {
    return c ? c->eng.load_state(c->slot, buf, bytes) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_device_bytes(flexrt_ctx *c, int64_t *bytes) {
    if (!c || !bytes) return FLEXRT_E_INVALID;
    *bytes = c->eng.device_bytes();
    return FLEXRT_OK;
}
extern "C" flexrt_status flexrt_profile(flexrt_ctx *c, int32_t enable) {
    return c ? c->eng.profile(enable != 0) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_get_kernel_times(flexrt_ctx *c, double ms[4], int64_t launches[4],
                                                 int64_t march_rays[1]) {
    if (!c || !ms || !launches) return FLEXRT_E_INVALID;
    return c->eng.kernel_times(ms, launches, march_rays);
}
extern "C" flexrt_status flexrt_set_launch(flexrt_ctx *c, int32_t agg, int32_t minb, int32_t blocks_per_sm,
                                           int32_t threads, int32_t slab) {
    return c ? c->eng.set_launch(agg, minb, blocks_per_sm, threads, slab) : FLEXRT_E_INVALID;
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
    b->merge_l_max = -1;
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
    cfg.merge_l_max = bc->merge_l_max;
    cfg.gen_capable = bc->gen_capable != 0;
    cfg.device_bytes_max = bc->device_bytes_max;
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
extern "C" flexrt_status flexrt_batch_get_segment_counts(flexrt_batch *b, int32_t slot, int32_t *out) {
    return b ? b->eng.segment_counts(slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_budget(flexrt_batch *b, int32_t slot, double out[4]) {
    return b ? b->eng.budget(slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_screen_excess(flexrt_batch *b, int32_t slot, double *photons) {
    return b ? b->eng.screen_excess(slot, photons) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_counts(flexrt_batch *b, int32_t slot, int64_t out[6]) {
    return b ? b->eng.counts(slot, out) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_rays(flexrt_batch *b, int32_t slot, int64_t cap, int32_t *level,
                                               int64_t *pixel, int32_t *emitter, int32_t *birth, int32_t *dir,
                                               double *photons, int64_t *n) {
    return b ? b->eng.rays(slot, cap, level, pixel, emitter, birth, dir, photons, n) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_ionized_volume(flexrt_batch *b, int32_t slot, double *x_ion) {
    return b ? b->eng.ionized_volume(slot, x_ion) : FLEXRT_E_INVALID;
}
extern "C" flexrt_status flexrt_batch_get_rays_merged(flexrt_batch *b, int32_t slot, int64_t cap, int32_t *merged,
                                                      int32_t *vertex, int32_t *dist, int64_t *pos, double *thr,
                                                      int64_t *n) {
    return b ? b->eng.rays_merged(slot, cap, merged, vertex, dist, pos, thr, n) : FLEXRT_E_INVALID;
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
extern "C" flexrt_status flexrt_batch_set_launch(flexrt_batch *b, int32_t agg, int32_t minb, int32_t bps,
                                                 int32_t threads, int32_t slab) {
    return b ? b->eng.set_launch(agg, minb, bps, threads, slab) : FLEXRT_E_INVALID;
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

extern "C" flexrt_status flexrt_probe_rates(int64_t n, const float *T, float *out) {
    if (n < 0 || (n && (!T || !out))) return FLEXRT_E_INVALID;
    for (int64_t i = 0; i < n; ++i)
        if (!(T[i] >= 1.0f && T[i] <= 1.0e9f)) return FLEXRT_E_INVALID;
    if (n == 0) return FLEXRT_OK;
    DevBuf<float> dT, dout;
    if (dT.alloc(n) != cudaSuccess || dout.alloc(4 * n) != cudaSuccess) return FLEXRT_E_OOM;
    if (cudaMemcpy(dT.p, T, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return FLEXRT_E_CUDA;
    if (launch_probe_rates(n, dT.p, dout.p, 0) != cudaSuccess) return FLEXRT_E_CUDA;
    if (cudaMemcpy(out, dout.p, 4 * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return FLEXRT_E_CUDA;
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

extern "C" flexrt_status flexrt_probe_merge_pixel(int32_t level, int64_t n, const int32_t *d, const int32_t *Rq,
                                                  int64_t n_rot, int32_t *out) {
    if (level < 0 || level > FLEXRT_MAX_LEVEL || n < 0 || !Rq || (n && (!d || !out)) || !(n_rot == 1 || n_rot == n))
        return FLEXRT_E_INVALID;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (d[i] > (1 << 21) || d[i] < -(1 << 21)) return FLEXRT_E_INVALID;
    for (int64_t k = 0; k < 9 * n_rot; ++k)
        if (Rq[k] > (1 << 24) || Rq[k] < -(1 << 24)) return FLEXRT_E_INVALID;
    DevBuf<int32_t> dd, dr;
    DevBuf<uint32_t> dout;
    if (dd.alloc(3 * n) != cudaSuccess || dr.alloc(9 * n_rot) != cudaSuccess || dout.alloc(n) != cudaSuccess)
        return FLEXRT_E_OOM;
    if (cudaMemcpy(dd.p, d, 3 * n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dr.p, Rq, 9 * n_rot * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return FLEXRT_E_CUDA;
    if (launch_probe_merge_pixel(level, n, dd.p, dr.p, n_rot > 1, dout.p, 0) != cudaSuccess) return FLEXRT_E_CUDA;
    if (cudaMemcpy(out, dout.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return FLEXRT_E_CUDA;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_probe_merge(const flexrt_merge_probe *p, int64_t n, const flexrt_probe_rays *in,
                                           int64_t cap, flexrt_probe_rays *out, int64_t *n_out) {
    if (!p || !in || !out || !n_out || n < 0 || cap < 0) return free_fail(FLEXRT_E_INVALID, "probe_merge: null");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 1000 || p->ny > 1000 || p->nz > 1000 || p->nbins < 1 ||
        p->nbins > FLEXRT_MAX_BINS || p->l_merge < 0 || p->l_merge > 11 || p->l_src < 0 || p->l_max > 12 ||
        p->l_max < p->l_src || p->k_ex < 0 || p->n_emitters < 0 || (p->n_emitters && (!p->emitter_cell || !p->emitter_n0)))
        return free_fail(FLEXRT_E_INVALID, "probe_merge: bad constants");
    if (n && (!in->pixlev || !in->emitter || !in->birth || !in->dir || !in->photons || !in->pos || !in->aux || !in->thr))
        return free_fail(FLEXRT_E_INVALID, "probe_merge: null ray array");
    if (cap && (!out->pixlev || !out->emitter || !out->birth || !out->dir || !out->photons || !out->pos || !out->aux ||
                !out->thr))
        return free_fail(FLEXRT_E_INVALID, "probe_merge: null output array");
    const long long ncell = (long long)p->nx * p->ny * p->nz;
    const int nb = p->nbins, ndir = 12 << (2 * p->l_merge);
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t e = in->emitter[i];
        const bool mg = (e & 0x80000000u) != 0;
        if (mg ? (long long)(e & 0x7fffffffu) >= ncell : (int32_t)e >= p->n_emitters)
            return free_fail(FLEXRT_E_INVALID, "probe_merge: emitter out of range");
        if ((in->pixlev[i] >> 28) > (uint32_t)p->l_max || (mg && (in->aux[i] & 0x7fff0000u)))
            return free_fail(FLEXRT_E_INVALID, "probe_merge: bad level or aux word");
        for (int a = 0; a < 3; ++a)
            if (in->dir[3 * i + a] > (1 << 21) || in->dir[3 * i + a] < -(1 << 21))
                return free_fail(FLEXRT_E_INVALID, "probe_merge: direction out of range");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int4 *tab = nullptr;
    const int lt = p->l_merge;
    if (get_pixtab(dev, lt, 0, &tab) != cudaSuccess) return free_fail(FLEXRT_E_CUDA, "probe_merge: pixel table");
    // one simulation (slot 0) whose march left the n rays in queue 1
    SimDev h;
    std::memset(&h, 0, sizeof(h));
    h.nx = p->nx; h.ny = p->ny; h.nz = p->nz; h.nb = nb;
    h.ncell = ncell;
    h.l_src = p->l_src; h.l_max = p->l_max;
    h.active = 1; h.step = p->step; h.rotate = p->rotate; h.seed = p->seed; h.eps_term = p->eps_term;
    h.merge = 1; h.l_merge = p->l_merge; h.ndir = ndir; h.k_ex = p->k_ex;
    SimAcc acc;
    std::memset(&acc, 0, sizeof(acc));
    acc.p_rays_out = (double)n;
    Ctl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.par = 0; ctl.cnt[1] = n; ctl.n_ranges = 1; ctl.ncell_active = ncell;
    // the queue holds the n rays and the merged rays appended after them
    // (each stands for two or more of the n)
    const long long m = std::max<long long>(n, 1), mq = m + m / 2 + 1;
    // per-block lists of the merge passes: each block's run starts at a
    // multiple of 256 past its first queue slot
    const long long ml = m + (long long)MERGE_MAX_BLOCKS * 256;
    const int gw = 12 + 4 * ((nb + 4) / 4);
    DevBuf<Ctl> dctl;
    DevBuf<SimDev> dsim;
    DevBuf<SimAcc> dacc;
    DevBuf<uint32_t> qpl[2], qem[2], qma[2], hist, sel, tkey, cand, ckey, lead_slot, bcnt, bled;
    DevBuf<uint4> tgrp, gcm;
    DevBuf<int32_t> qbi[2], qd[2], qm[2], tsim, rsim, lead_sim;
    DevBuf<float> qph[2], qthr[2], grp, n0;
    DevBuf<int4> ecell, rot;
    DevBuf<long long> pref, cell0;
    bool ok = dctl.alloc(1) == cudaSuccess && dsim.alloc(1) == cudaSuccess && dacc.alloc(1) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
        ok = qpl[k].alloc(mq) == cudaSuccess && qem[k].alloc(mq) == cudaSuccess && qma[k].alloc(mq) == cudaSuccess &&
             qbi[k].alloc(mq) == cudaSuccess && qd[k].alloc(3 * mq) == cudaSuccess && qm[k].alloc(3 * mq) == cudaSuccess &&
             qph[k].alloc(nb * mq) == cudaSuccess && qthr[k].alloc(mq) == cudaSuccess;
    ok = ok && hist.alloc(HIST_BINS) == cudaSuccess && sel.alloc(8) == cudaSuccess && tkey.alloc(m) == cudaSuccess &&
         tsim.alloc(m) == cudaSuccess && gcm.alloc(ncell * ndir) == cudaSuccess && tgrp.alloc(ml) == cudaSuccess &&
         cand.alloc(ml) == cudaSuccess && ckey.alloc(ml) == cudaSuccess && bcnt.alloc(MERGE_MAX_BLOCKS) == cudaSuccess &&
         bled.alloc(MERGE_MAX_BLOCKS) == cudaSuccess &&
         grp.alloc(ncell * ndir * gw) == cudaSuccess && rot.alloc(3 * ncell) == cudaSuccess &&
         ecell.alloc(std::max(p->n_emitters, 1)) == cudaSuccess && n0.alloc(std::max(p->n_emitters, 1)) == cudaSuccess &&
         pref.alloc(2) == cudaSuccess && cell0.alloc(1) == cudaSuccess && rsim.alloc(1) == cudaSuccess &&
         lead_slot.alloc(ml) == cudaSuccess && lead_sim.alloc(ml) == cudaSuccess;
    if (!ok) return free_fail(FLEXRT_E_OOM, "probe_merge: device allocation failed");
    // queue layout: structure of arrays, photons bin-major
    auto queue = [&](int k) {
        Queue q{};
        q.pl = qpl[k].p; q.em = qem[k].p; q.bi = qbi[k].p;
        q.dx = qd[k].p; q.dy = qd[k].p + mq; q.dz = qd[k].p + 2 * mq;
        for (int b = 0; b < nb; ++b) q.ph[b] = qph[k].p + b * mq;
        q.mx = qm[k].p; q.my = qm[k].p + mq; q.mz = qm[k].p + 2 * mq;
        q.ma = qma[k].p; q.mthr = qthr[k].p;
        return q;
    };
    const Queue q0 = queue(0), q1 = queue(1);
    std::vector<int32_t> d3(3 * mq), m3(3 * mq);
    std::vector<float> ph(nb * mq);
    std::vector<uint32_t> ma(mq);
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) { d3[a * mq + i] = in->dir[3 * i + a]; m3[a * mq + i] = in->pos[3 * i + a]; }
        for (int b = 0; b < nb; ++b) ph[b * mq + i] = in->photons[(size_t)nb * i + b];
        ma[i] = in->aux[i] & 0x8000ffffu;              // simulation 0
    }
    std::vector<int4> ec(std::max(p->n_emitters, 1));
    for (int k = 0; k < p->n_emitters; ++k)
        ec[k] = make_int4(p->emitter_cell[3 * k], p->emitter_cell[3 * k + 1], p->emitter_cell[3 * k + 2], 0);
    const long long pr[2] = {0, ncell}, c0 = 0;
    const int32_t s0 = 0;
    auto up = [](void *dst, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    ok = up(dctl.p, &ctl, sizeof(ctl)) && up(dsim.p, &h, sizeof(h)) && up(dacc.p, &acc, sizeof(acc)) &&
         up(q1.pl, in->pixlev, n * 4) && up(q1.em, in->emitter, n * 4) && up(q1.bi, in->birth, n * 4) &&
         up(qd[1].p, d3.data(), 3 * mq * 4) && up(qm[1].p, m3.data(), 3 * mq * 4) &&
         up(qph[1].p, ph.data(), nb * mq * 4) && up(q1.ma, ma.data(), mq * 4) && up(q1.mthr, in->thr, n * 4) && up(ecell.p, ec.data(), ec.size() * sizeof(int4)) &&
         up(n0.p, p->emitter_n0, p->n_emitters * sizeof(float)) && up(pref.p, pr, sizeof(pr)) &&
         up(cell0.p, &c0, sizeof(c0)) && up(rsim.p, &s0, sizeof(s0));
    ok = ok && cudaMemset(hist.p, 0, HIST_BINS * 4) == cudaSuccess && cudaMemset(sel.p, 0, 32) == cudaSuccess &&
         cudaMemset(gcm.p, 0, ncell * ndir * 16) == cudaSuccess &&
         cudaMemset(grp.p, 0, (size_t)ncell * ndir * gw * 4) == cudaSuccess;
    if (!ok) return free_fail(FLEXRT_E_CUDA, "probe_merge: upload failed");
    Emitters em{};
    em.cell = ecell.p; em.n0 = n0.p;
    Ranges rg{pref.p, cell0.p, rsim.p};
    MergeWork w{};
    w.hist = hist.p; w.sel = sel.p; w.tkey = tkey.p; w.tsim = tsim.p;
    w.grp = grp.p; w.gcm = gcm.p; w.cand = cand.p; w.ckey = ckey.p; w.tgrp = tgrp.p; w.rot = rot.p; w.ndir = ndir;
    w.grp_w = gw; w.hrep = 1; w.lead_slot = lead_slot.p; w.lead_sim = lead_sim.p;
    w.bcnt = bcnt.p; w.bled = bled.p; w.lead_cap = ml;
    MergeArgs a{dctl.p, dsim.p, dacc.p, 1, {q0, q1}, em, rg, tab, lt, w, nb, mq};
    if (launch_merge(a, sms, 0, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return free_fail(FLEXRT_E_CUDA, "probe_merge: kernels failed");
    Ctl hc;
    if (cudaMemcpy(&hc, dctl.p, sizeof(hc), cudaMemcpyDeviceToHost) != cudaSuccess)
        return free_fail(FLEXRT_E_CUDA, "probe_merge: read-back failed");
    // the rays stay in queue 1; the merge leaves holes where its groups'
    // members were (skipped here) and appends the merged rays
    const int k = 1;
    const long long cnt = std::min<long long>(hc.cnt[1], mq);
    std::vector<uint32_t> opl(mq), oem(mq), oma(mq);
    std::vector<int32_t> obi(mq), od(3 * mq), om(3 * mq);
    std::vector<float> oph(nb * mq), othr(mq);
    auto down = [](void *dst, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    const Queue qq = k ? q1 : q0;
    ok = down(opl.data(), qq.pl, mq * 4) && down(oem.data(), qq.em, mq * 4) && down(obi.data(), qq.bi, mq * 4) &&
         down(od.data(), qd[k].p, 3 * mq * 4) && down(om.data(), qm[k].p, 3 * mq * 4) &&
         down(oph.data(), qph[k].p, nb * mq * 4) && down(oma.data(), qq.ma, mq * 4) && down(othr.data(), qq.mthr, mq * 4);
    if (!ok) return free_fail(FLEXRT_E_CUDA, "probe_merge: read-back failed");
    long long o = 0;
    for (long long i = 0; i < cnt; ++i) {
        if (opl[i] == DEAD_RAY) continue;
        if (o < cap) {
            const bool mg = (oem[i] & 0x80000000u) != 0;
            out->pixlev[o] = opl[i];
            out->emitter[o] = oem[i];
            out->birth[o] = obi[i];
            for (int a2 = 0; a2 < 3; ++a2) {
                out->dir[3 * o + a2] = od[a2 * mq + i];
                out->pos[3 * o + a2] = mg ? om[a2 * mq + i] : 0;
            }
            for (int b = 0; b < nb; ++b) out->photons[(size_t)nb * o + b] = oph[b * mq + i];
            out->aux[o] = mg ? (oma[i] & 0x8000ffffu) : 0u;
            out->thr[o] = mg ? othr[i] : 0.0f;
        }
        ++o;
    }
    *n_out = o;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_probe_traverse(int64_t n, const int64_t *p0, const int32_t *dir,
                                               const flexrt_grid *g, int32_t *cells, float *ds, int32_t *nseg,
                                               int32_t *escaped) {
    if (n < 0 || !g || (n && (!p0 || !dir || !cells || !ds || !nseg || !escaped))) return FLEXRT_E_INVALID;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (dir[i] > (1 << 21) || dir[i] < -(1 << 21) || p0[i] > (1LL << 31) - (1LL << 22) ||
            p0[i] < -(1LL << 31) + (1LL << 22))
            return FLEXRT_E_INVALID;
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
