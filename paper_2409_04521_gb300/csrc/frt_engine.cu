// frt_engine.cu -- host engine: device arenas, simulation slots, step launch
// (direct or replayed from a CUDA graph), accounting and read-back.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "frt_engine.h"

namespace frt {

namespace {

constexpr double EV_ERG = 1.602176634e-12;

// Generalized mode: atoms of a whole cell per unit n_H, in code photons,
// (1 + chi) V / nref, in single precision (capped at the largest float)
static float atoms_per_nH(const frt::SimDev &h) {
    const double v = (1.0 + h.chi) * h.dx_phys * h.dx_phys * h.dx_phys / h.nref;
    return v < 3.0e38 ? (float)v : 3.0e38f;
}
constexpr double MYR_S = 3.15576e13;

// process-wide fixed-point pixel vector tables, one per device, grown on demand
struct PixTable {
    int4 *ptr = nullptr;
    int level = -1;
};
std::mutex g_tab_mu;
std::map<int, PixTable> g_tabs;

void split_table(double nmin, int32_t *K) {
    const double f = std::sqrt(3.0 / (M_PI * nmin));
    for (int l = 0; l < 16; ++l) {
        long long k = (long long)std::ceil(std::ldexp(f, l));
        if (k < 1) k = 1;
        if (k > (1LL << 30)) k = 1LL << 30;
        K[l] = (int32_t)k;
    }
}

int ring_length(int n) { return (int)std::ceil(std::sqrt(3.0) * n) + 4; }

// queue bytes per ray slot; merged rays add position, distance word and threshold
size_t ray_bytes(int nb, bool merge) { return 6 * sizeof(int32_t) + (size_t)nb * sizeof(float) + (merge ? 20 : 0); }

}  // namespace

cudaError_t get_pixtab(int device, int level, cudaStream_t st, const int4 **out) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    PixTable &t = g_tabs[device];
    if (t.level < level) {
        int4 *p = nullptr;
        const size_t bytes = (size_t)(4LL * ((1LL << (2 * (level + 1))) - 1)) * sizeof(int4);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return e;
        e = launch_pixtab(p, level, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { cudaFree(p); return e; }
        if (t.ptr) cudaFree(t.ptr);
        t.ptr = p;
        t.level = level;
    }
    *out = t.ptr;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
void RangeAllocator::reset(long long capacity) {
    cap_ = capacity;
    used_ = 0;
    free_.clear();
    if (capacity > 0) free_.push_back({0, capacity});
}
long long RangeAllocator::alloc(long long n) {
    if (n <= 0) return -1;
    for (size_t i = 0; i < free_.size(); ++i) {
        if (free_[i].n >= n) {
            const long long s = free_[i].start;
            free_[i].start += n;
            free_[i].n -= n;
            if (free_[i].n == 0) free_.erase(free_.begin() + (long)i);
            used_ += n;
            return s;
        }
    }
    return -1;
}
void RangeAllocator::release(long long start, long long n) {
    if (n <= 0) return;
    used_ -= n;
    auto it = std::lower_bound(free_.begin(), free_.end(), start,
                               [](const Free &f, long long v) { return f.start < v; });
    it = free_.insert(it, {start, n});
    // merge with neighbours
    size_t i = (size_t)(it - free_.begin());
    if (i + 1 < free_.size() && free_[i].start + free_[i].n == free_[i + 1].start) {
        free_[i].n += free_[i + 1].n;
        free_.erase(free_.begin() + (long)i + 1);
    }
    if (i > 0 && free_[i - 1].start + free_[i - 1].n == free_[i].start) {
        free_[i - 1].n += free_[i].n;
        free_.erase(free_.begin() + (long)i);
    }
}

// ---------------------------------------------------------------------------
flexrt_status Engine::cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FLEXRT_OK;
    err_ = std::string(what) + ": " + cudaGetErrorString(e);
    return FLEXRT_E_CUDA;
}

// Device allocations of the engine: counted against the context's cap
// (device_bytes_max; 0 = none); an allocation beyond it fails like a
// cudaMalloc that found no memory.
cudaError_t Engine::dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (cfg_.device_bytes_max > 0 && (long long)(alloc_bytes_ + bytes) > cfg_.device_bytes_max)
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    alloc_sizes_[*p] = bytes;
    alloc_bytes_ += bytes;
    return cudaSuccess;
}
void Engine::dev_free(void *p) {
    if (!p) return;
    auto it = alloc_sizes_.find(p);
    if (it != alloc_sizes_.end()) {
        alloc_bytes_ -= it->second;
        alloc_sizes_.erase(it);
    }
    cudaFree(p);
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return cuda(e__, #call);  \
    } while (0)

Engine::~Engine() {
    if (st_) cudaStreamSynchronize(st_);
    if (graph_) cudaGraphExecDestroy(graph_);
    // every device allocation of the engine, whether or not init completed
    for (auto &kv : alloc_sizes_) cudaFree(kv.first);
    alloc_sizes_.clear();
    if (h_err_) cudaFreeHost(h_err_);
    if (h_stage_) cudaFreeHost(h_stage_);
    if (h_nh_) cudaFreeHost(h_nh_);
    if (h_fields_) cudaFreeHost(h_fields_);
    if (ev_nh_) cudaEventDestroy(ev_nh_);
    if (ev_err_) cudaEventDestroy(ev_err_);
    if (ev_stage_) cudaEventDestroy(ev_stage_);
    for (auto e : ev_pool_) cudaEventDestroy(e);
    for (auto &v : ev_k_)
        for (auto &p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    if (mside_.fork) cudaEventDestroy(mside_.fork);
    if (mside_.join) cudaEventDestroy(mside_.join);
    if (mside_.st) cudaStreamDestroy(mside_.st);
    if (own_stream_ && st_) cudaStreamDestroy(st_);
}

flexrt_status Engine::init(const EngineConfig &cfg) {
    cfg_ = cfg;
    if (cfg_.nb < 1 || cfg_.nb > MAXB || cfg_.max_sims < 1 || cfg_.max_sims > 512 || cfg_.cell_capacity < 1 ||
        cfg_.max_grid < 1 || cfg_.max_grid > 1000)
        return fail(FLEXRT_E_INVALID, "bad engine configuration");
    CK(cudaGetDevice(&device_));
    if (cfg_.stream) st_ = (cudaStream_t)cfg_.stream;
    else {
        CK(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
        own_stream_ = true;
    }
    em_.ring_w = ring_length(cfg_.max_grid);
    int32_t K[16];
    split_table(cfg_.n_ray_min, K);
    int L = 0;
    while (L < cfg_.l_max && K[L] <= em_.ring_w) ++L;
    ltab_ = std::min(L, 11);

    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const bool mrg = cfg_.merge_l_max >= 0;
    if (cfg_.merge_l_max > 11) return fail(FLEXRT_E_INVALID, "merge level above 11");
    long long cap = cfg_.ray_capacity;
    if (cap <= 0) cap = std::min((long long)(0.3 * (double)freeb / (2.0 * ray_bytes(cfg_.nb, mrg))), 1600000000LL);
    cfg_.ray_capacity = cap = std::max(cap, 1024LL);
    // queue slots beyond the live-ray capacity for the unused tails of the
    // march's warp-private output runs
    cap += cap / 4 + 4096;
    // the kernels index the queue with 32-bit integers
    if (cap >= (1LL << 31) - (1LL << 24)) return fail(FLEXRT_E_INVALID, "ray capacity above the 32-bit queue index");
    qcap_ = cap;

    // ray queues: one allocation, structure of arrays, two buffers
    {
        // each array starts on a 256-byte boundary (vector loads of the queue)
        const size_t a = ((size_t)cap * 4 + 255) & ~(size_t)255, per = a * (ray_bytes(cfg_.nb, mrg) / 4);
        char *base = nullptr;
        if (dev_alloc((void **)&base, 2 * per + 256) != cudaSuccess) return fail(FLEXRT_E_OOM, "ray queue allocation failed");
        qmem_ = base;
        for (int k = 0; k < 2; ++k) {
            char *p = base + k * per;
            q_[k].pl = (uint32_t *)p; p += a;
            q_[k].em = (uint32_t *)p; p += a;
            q_[k].bi = (int32_t *)p; p += a;
            q_[k].dx = (int32_t *)p; p += a;
            q_[k].dy = (int32_t *)p; p += a;
            q_[k].dz = (int32_t *)p; p += a;
            for (int b = 0; b < MAXB; ++b) {
                q_[k].ph[b] = b < cfg_.nb ? (float *)p : nullptr;
                if (b < cfg_.nb) p += a;
            }
            if (mrg) {
                q_[k].mx = (int32_t *)p; p += a;
                q_[k].my = (int32_t *)p; p += a;
                q_[k].mz = (int32_t *)p; p += a;
                q_[k].ma = (uint32_t *)p; p += a;
                q_[k].mthr = (float *)p; p += a;
            }
        }
    }
    const long long nc = cfg_.cell_capacity;
    const int ms = cfg_.max_sims;
#define ALLOC(ptr, n)                                                          \
    if (dev_alloc((void **)&(ptr), (size_t)(n) * sizeof(*(ptr))) != cudaSuccess) \
        return fail(FLEXRT_E_OOM, "device allocation failed: " #ptr)
    ALLOC(ctl_, 1);
    ALLOC(sims_, ms);
    ALLOC(acc_, ms);
    ALLOC(cells_.nH, nc);
    ALLOC(cells_.nHf, nc);
    ALLOC(cells_.y, nc);
    ALLOC(cells_.x, nc);
    ALLOC(cells_.T, nc);
    ALLOC(cells_.gamma, nc);
    ALLOC(cells_.kap, nc);
    ALLOC(cells_.dep, nc);
    if (cfg_.keep_diagnostics) ALLOC(cells_.segcnt, nc);
    ALLOC(cells_.xion, nc);
    ALLOC(cells_.rho, nc);
    ALLOC(cells_.fscr, nc);
    ALLOC(rg_.pref, ms + 1);
    ALLOC(rg_.cell0, ms);
    ALLOC(rg_.sim, ms);
#undef ALLOC
    if (mrg) {
        // merge scratch (Sec. 3.3): histograms and selections per slot, rank
        // content / simulation per queue slot, group sums, sizes, largest
        // contents and leaders per (cell, merge pixel), rotation rows per
        // cell, the per-block candidate and merged-ray lists (a block's run
        // starts at a multiple of 256 past its first queue slot) and counts
        mw_.ndir = 12 << (2 * cfg_.merge_l_max);
        mw_.grp_w = 12 + 4 * ((cfg_.nb + 4) / 4);   // 6 integer sums, photons and threshold
        const long long ngrp = nc * (long long)mw_.ndir;
        if (ngrp >= (1LL << 31)) return fail(FLEXRT_E_INVALID, "cells x merge directions must stay below 2^31");
        mw_.hrep = std::max(1, std::min(32, 64 / ms));
        mw_.lead_cap = cap + (long long)MERGE_MAX_BLOCKS * 256;
        const size_t nl = (size_t)mw_.lead_cap;
        const size_t sz[] = {(size_t)ms * mw_.hrep * HIST_BINS * 4, (size_t)ms * 32, (size_t)cap * 4,
                             (size_t)cap * 4, (size_t)ngrp * mw_.grp_w * 4, (size_t)ngrp * 16,
                             (size_t)nc * 48, nl * 4, nl * 4, nl * 4, nl * 4, nl * 16,
                             (size_t)MERGE_MAX_BLOCKS * 4, (size_t)MERGE_MAX_BLOCKS * 4};
        size_t tot = 0;
        for (size_t v : sz) tot += (v + 255) & ~(size_t)255;
        if (dev_alloc(&mwmem_, tot) != cudaSuccess) return fail(FLEXRT_E_OOM, "merge scratch allocation failed");
        char *p = (char *)mwmem_;
        void **dst[] = {(void **)&mw_.hist, (void **)&mw_.sel, (void **)&mw_.tkey, (void **)&mw_.tsim,
                        (void **)&mw_.grp, (void **)&mw_.gcm, (void **)&mw_.rot, (void **)&mw_.cand,
                        (void **)&mw_.ckey, (void **)&mw_.lead_slot, (void **)&mw_.lead_sim, (void **)&mw_.tgrp,
                        (void **)&mw_.bcnt, (void **)&mw_.bled};
        static_assert(sizeof(sz) / sizeof(sz[0]) == sizeof(dst) / sizeof(dst[0]), "merge scratch layout");
        for (size_t k = 0; k < sizeof(sz) / sizeof(sz[0]); ++k) { *dst[k] = p; p += (sz[k] + 255) & ~(size_t)255; }
        if (cap >= (1LL << 32)) return fail(FLEXRT_E_INVALID, "merging needs fewer than 2^32 queue slots");
        CK(cudaMemsetAsync(mwmem_, 0, tot, st_));
        CK(cudaStreamCreateWithFlags(&mside_.st, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&mside_.fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&mside_.join, cudaEventDisableTiming));
    }
    if (cudaMallocHost(&h_err_, 64) != cudaSuccess) return fail(FLEXRT_E_OOM, "pinned allocation failed");
    if (ms > 1) {
        // members are admitted while others step: their densities go up
        // through pinned staging, so that admission does not wait for the GPU
        const size_t nh = (size_t)cfg_.max_grid * cfg_.max_grid * cfg_.max_grid * sizeof(double);
        if (cudaMallocHost(&h_nh_, nh) != cudaSuccess) return fail(FLEXRT_E_OOM, "pinned allocation failed");
        CK(cudaEventCreateWithFlags(&ev_nh_, cudaEventDisableTiming));
    }
    if (cudaMallocHost(&h_stage_, (size_t)(ms + 1) * 6 * sizeof(double)) != cudaSuccess)
        return fail(FLEXRT_E_OOM, "pinned allocation failed");
    CK(cudaEventCreateWithFlags(&ev_err_, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_stage_, cudaEventDisableTiming));
    cell_alloc_.reset(nc);
    em_cap_ = 0;
    flexrt_status s = grow_emitters(std::max(cfg_.emitter_capacity, 16));
    if (s != FLEXRT_OK) return s;
    em_alloc_.reset(em_cap_);
    slots_.assign(ms, Slot());

    CK(cudaMemsetAsync(ctl_, 0, sizeof(Ctl), st_));
    CK(cudaMemsetAsync(sims_, 0, (size_t)ms * sizeof(SimDev), st_));
    CK(cudaMemsetAsync(acc_, 0, (size_t)ms * sizeof(SimAcc), st_));
    cudaError_t e = get_pixtab(device_, ltab_, st_, &pixtab_);
    if (e != cudaSuccess) return cuda(e, "pixel table");

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device_);
    sm_count_ = std::max(sms, 1);
    const int ext = ext_variants();
    if (!march_variant_exists(cfg_.nb, march_agg_, march_minb_, ext)) { march_agg_ = 0; march_minb_ = 2; }
    CK(march_prepare(cfg_.nb, march_agg_, march_minb_, ms, ext));
    const int per_sm = march_max_blocks_per_sm(cfg_.nb, march_agg_, march_minb_, march_threads_, ms, ext);
    if (per_sm < 1) return fail(FLEXRT_E_INVALID, "too many simulation slots for one march block");
    march_blocks_ = sm_count_ * std::max(per_sm, 1);
    chem_blocks_ = (int)std::max<long long>(1, std::min<long long>((nc + 255) / 256, (long long)sm_count_ * 8));
    CK(cudaStreamSynchronize(st_));
    return FLEXRT_OK;
}

flexrt_status Engine::grow_emitters(int need) {
    if (need <= em_cap_) return FLEXRT_OK;
    if (em_cap_ > 0 && cfg_.emitter_capacity > 0)
        return fail(FLEXRT_E_CAPACITY, "emitter table full");
    const int cap = std::max(need, std::max(16, 2 * em_cap_));
    Emitters ne{};
    ne.ring_w = em_.ring_w;
    if (dev_alloc((void **)&ne.cell, cap * sizeof(int4)) != cudaSuccess ||
        dev_alloc((void **)&ne.local, cap * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc((void **)&ne.ndot, cap * sizeof(double)) != cudaSuccess ||
        dev_alloc((void **)&ne.n0, cap * sizeof(float)) != cudaSuccess ||
        dev_alloc((void **)&ne.ring, (size_t)cap * ne.ring_w * 3 * sizeof(int4)) != cudaSuccess ||
        dev_alloc((void **)&ne.act, cap * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc((void **)&ne.act_off, cap * sizeof(long long)) != cudaSuccess) {
        dev_free(ne.cell); dev_free(ne.local); dev_free(ne.ndot); dev_free(ne.n0);
        dev_free(ne.ring); dev_free(ne.act); dev_free(ne.act_off);
        return fail(FLEXRT_E_OOM, "emitter table allocation failed");
    }
    if (em_cap_ > 0) {
        CK(cudaStreamSynchronize(st_));
        CK(cudaMemcpy(ne.cell, em_.cell, em_cap_ * sizeof(int4), cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(ne.local, em_.local, em_cap_ * sizeof(int32_t), cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(ne.ndot, em_.ndot, em_cap_ * sizeof(double), cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(ne.n0, em_.n0, em_cap_ * sizeof(float), cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(ne.ring, em_.ring, (size_t)em_cap_ * ne.ring_w * 3 * sizeof(int4), cudaMemcpyDeviceToDevice));
    }
    dev_free(em_.cell); dev_free(em_.local); dev_free(em_.ndot); dev_free(em_.n0);
    dev_free(em_.ring); dev_free(em_.act); dev_free(em_.act_off);
    em_ = ne;
    em_cap_ = cap;
    emit_blocks_ = std::max(1, std::min((em_cap_ + 127) / 128, 1024));
    graph_dirty_ = true;
    return FLEXRT_OK;
}

flexrt_status Engine::make_sim(const flexrt_grid *grid, const flexrt_box *box, const double *n_H,
                               const flexrt_mfp *mfp, const flexrt_spectrum *sp, const flexrt_options *opt_in,
                               SimDev &h, std::string &err) {
    if (!grid || !box || !n_H || !sp) { err = "null argument"; return FLEXRT_E_INVALID; }
    flexrt_options opt;
    if (opt_in) opt = *opt_in; else flexrt_default_options(&opt);
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nx > 1000 || grid->ny > 1000 || grid->nz > 1000) {
        err = "grid must be 1..1000 cells per axis"; return FLEXRT_E_INVALID;
    }
    if (sp->nbins < 1 || sp->nbins > FLEXRT_MAX_BINS || !sp->frac || !sp->sigma_cm2 || !sp->eheat_erg) {
        err = "bad spectrum"; return FLEXRT_E_INVALID;
    }
    if (opt.l_src < 0 || opt.l_max < opt.l_src || opt.l_max > FLEXRT_MAX_LEVEL || !(opt.n_ray_min > 0) ||
        opt.chem_iters < 1 || !(box->box_cm_comoving > 0) || box->redshift <= -1.0) {
        err = "bad options or box"; return FLEXRT_E_INVALID;
    }
    std::memset(&h, 0, sizeof(h));
    h.nx = grid->nx; h.ny = grid->ny; h.nz = grid->nz; h.nb = sp->nbins;
    h.ncell = (long long)grid->nx * grid->ny * grid->nz;
    h.l_src = opt.l_src; h.l_max = opt.l_max;
    split_table(opt.n_ray_min, h.K);
    h.active = 1;
    h.rotate = opt.rotate ? 1 : 0;
    h.seed = opt.seed;
    h.eps_term = (float)opt.eps_term;
    h.sigma_ref = sp->sigma_cm2[0];
    if (!(h.sigma_ref > 0)) { err = "sigma of bin 0 must be positive"; return FLEXRT_E_INVALID; }
    for (int b = 0; b < sp->nbins; ++b) {
        h.sig[b] = (float)(sp->sigma_cm2[b] / h.sigma_ref);
        h.sige[b] = (float)(sp->sigma_cm2[b] / h.sigma_ref * sp->eheat_erg[b] / EV_ERG);
        h.eh[b] = (float)(sp->eheat_erg[b] / EV_ERG);
        h.frac[b] = (float)sp->frac[b];
    }
    h.dx_com = box->box_cm_comoving / grid->nx;
    h.dx_phys = h.dx_com / (1.0 + box->redshift);
    h.inv_ncast = 1.0 / (double)(12LL << (2 * opt.l_src));
    h.z = box->redshift;
    {
        const double kB = 1.380649e-16, sT = 6.6524587e-25, a = 7.5657e-15, me = 9.1093837e-28, cl = 2.99792458e10;
        const double Tc = 2.7255 * (1.0 + box->redshift);
        h.Tcmb = (float)Tc;
        h.compton_c = (float)(4.0 * kB * sT * a * Tc * Tc * Tc * Tc / (me * cl));
    }
    h.alpha_const = opt.alpha_B_const;
    h.rates = opt.rates; h.isothermal = opt.isothermal ? 1 : 0; h.chem_iters = opt.chem_iters;
    flexrt_mfp m{};
    if (mfp) m = *mfp;
    h.mfp_mode = m.mode;
    h.lambda0_c = m.lambda0_cm_comoving; h.delta_exp = m.delta_exp; h.gamma_ref = m.gamma_ref;
    h.gamma_exp = m.gamma_exp; h.gamma_floor = m.gamma_floor; h.xion_thr = m.xion_threshold;
    if ((m.mode == 1 || m.mode == 2) && !(m.lambda0_cm_comoving > 0)) { err = "lambda0 must be positive"; return FLEXRT_E_INVALID; }
    if (m.mode == 2 && !(m.gamma_ref > 0)) { err = "gamma_ref must be positive"; return FLEXRT_E_INVALID; }
    double mean = m.nH_mean;
    if (!(mean > 0)) {
        double s = 0.0;
        for (long long i = 0; i < h.ncell; ++i) s += n_H[i];
        mean = s / (double)h.ncell;
    }
    h.nH_mean = mean;
    h.ksc = h.sigma_ref * h.dx_phys;
    h.inv_nH_mean = mean > 0 ? 1.0 / mean : 0.0;
    h.inv_gamma_ref = m.gamma_ref > 0 ? 1.0 / m.gamma_ref : 0.0;
    h.y_thr = 1.0 - m.xion_threshold;
    h.kap_sub0 = m.lambda0_cm_comoving > 0 ? (float)(h.dx_com / m.lambda0_cm_comoving) : 0.0f;
    h.x_init = opt.x_init; h.T_init = opt.T_init;
    h.nref = 1.0;
    if (opt.gamma_iters < 1 || opt.gamma_iters > 64) { err = "gamma_iters must be 1..64"; return FLEXRT_E_INVALID; }
    h.gamma_iters = opt.gamma_iters;
    if (opt.gen_mode) {
        // Generalized Opacity mode (Sec. 4.2): lambda, Gamma and the screens'
        // shares are iterated (a screen first reached in the last pass takes
        // everything, and what exceeds its atoms is lost: 8e-3 of the photons
        // emitted with 3 passes, 6e-5 with 4, 2e-6 with 5 on a Stromgren test);
        // with evolving temperature, newly ionised gas enters at T_reion and
        // heats by the power-law law of Eq. 22, whose bracket -- the mean
        // excess energy per ionisation of J ~ nu^-alpha_pl cut at 4 Ryd with
        // sigma ~ nu^-2.75 -- is evaluated here once
        if (opt.gamma_iters < 4 || !(opt.chi >= 0.0)) {
            err = "Generalized mode needs gamma_iters >= 4 and chi >= 0"; return FLEXRT_E_INVALID;
        }
        if (!opt.isothermal && !(opt.t_reion > 0.0 && opt.t_reion < 1e9 && opt.alpha_pl > -1.0 && opt.alpha_pl < 20.0)) {
            err = "Generalized mode with evolving T needs 0 < t_reion < 1e9 and -1 < alpha_pl < 20"; return FLEXRT_E_INVALID;
        }
        h.gen_mode = 1;
        h.chi = opt.chi;
        const double s = opt.alpha_pl + 2.75;   // photons absorbed ~ e^-(s+1) de over e in [1, 4] Ryd
        h.t_reion = (float)opt.t_reion;
        h.pl_heat = (float)(13.6 * EV_ERG * (s / (s - 1.0) * (1.0 - std::pow(4.0, 1.0 - s)) / (1.0 - std::pow(4.0, -s)) - 1.0));
    }
    if (m.mode == 3 && !opt.gen_mode) { err = "mfp mode 3 is for Generalized mode"; return FLEXRT_E_INVALID; }
    if (opt.merge) {
        if (opt.l_merge < 0 || opt.l_merge > 11 || opt.l_merge > opt.l_max || !(opt.n_ex >= 0.0)) {
            err = "bad merge options (0 <= l_merge <= min(11, l_max), n_ex >= 0)"; return FLEXRT_E_INVALID;
        }
        h.merge = 1;
        h.l_merge = opt.l_merge;
        h.ndir = 12 << (2 * opt.l_merge);
        const double k = std::floor(opt.n_ex * (double)h.ncell);
        h.k_ex = k > 4e18 ? (long long)4e18 : (long long)k;
    }
    // an isothermal run evaluates its rate coefficients once (same fits as
    // the per-cell device evaluation, in double precision)
    {
        const double T = opt.T_init, lam = 2.0 * 157807.0 / T;
        const double aB = 2.753e-14 * std::pow(lam, 1.5) / std::pow(1.0 + std::pow(lam / 2.740, 0.407), 2.242);
        const double ci = lam > 180.0 ? 0.0
                                      : 21.11 * std::pow(T, -1.5) * std::exp(-0.5 * lam) * std::pow(lam, -1.089) /
                                            std::pow(1.0 + std::pow(lam / 0.354, 0.874), 1.101);
        h.alpha_iso = (float)(opt.rates ? aB : opt.alpha_B_const);
        h.coll_iso = (float)(opt.rates ? ci : 0.0);
    }
    {
        // single-precision copies for the chemistry kernel
        h.ksc_f = (float)h.ksc;
        h.inv_nH_mean_f = (float)h.inv_nH_mean;
        h.inv_gamma_ref_f = (float)h.inv_gamma_ref;
        h.neg_delta_exp_f = (float)(-h.delta_exp);
        h.gamma_exp_f = (float)h.gamma_exp;
        h.gamma_floor_f = (float)h.gamma_floor;
        float t = (float)h.y_thr;
        if ((double)t > h.y_thr) t = std::nextafter(t, -INFINITY);
        h.y_thr_dn = t;
        h.alpha_const_f = (float)h.alpha_const;
        h.chi_f = (float)h.chi;
        h.chi1_f = (float)(1.0 + h.chi);
        h.apn_f = atoms_per_nH(h);
    }
    return FLEXRT_OK;
}

flexrt_status Engine::add_sim(const SimDev &proto, const double *n_H, int *slot_out) {
    free_retired();
    const int ms = (int)slots_.size();
    int s = -1;
    for (int i = 0; i < ms; ++i)
        if (!slots_[i].used) { s = i; break; }
    if (s < 0) return fail(FLEXRT_E_CAPACITY, "no free simulation slot");
    const int edge = std::max(proto.nx, std::max(proto.ny, proto.nz));
    if (edge > cfg_.max_grid) return fail(FLEXRT_E_INVALID, "grid larger than the engine's max_grid");
    if (proto.nb > cfg_.nb) return fail(FLEXRT_E_INVALID, "more frequency bins than the engine's layout");
    if (proto.gen_mode && !cfg_.gen_capable)
        return fail(FLEXRT_E_INVALID, "engine not built for Generalized mode members");
    if (proto.merge && proto.l_merge > cfg_.merge_l_max)
        return fail(FLEXRT_E_INVALID, "merge level deeper than the engine's merge scratch allows");
    for (const Slot &o : slots_)
        if (o.used && o.h.gamma_iters != proto.gamma_iters)
            return fail(FLEXRT_E_INVALID, "members of one engine must use the same gamma_iters");
    const long long c0 = cell_alloc_.alloc(proto.ncell);
    if (c0 < 0) return fail(FLEXRT_E_CAPACITY, "cell arena full");
    Slot &sl = slots_[s];
    sl = Slot();
    sl.used = true;
    sl.active = true;
    sl.h = proto;
    sl.h.cell_off = c0;
    sl.h.ring_w = em_.ring_w;
    sl.h.step = 0;
    sl.h.active = 1;
    sl.cell0 = c0;
    // everything in stream order, behind the steps already enqueued (the
    // member's cells may be those of a member retired before them): the host
    // does not wait for the GPU
    CK(cudaMemcpyAsync(sims_ + s, &sl.h, sizeof(SimDev), cudaMemcpyHostToDevice, st_));
    CK(cudaMemsetAsync(acc_ + s, 0, sizeof(SimAcc), st_));
    const size_t nhb = (size_t)proto.ncell * sizeof(double);
    if (h_nh_ && nhb <= (size_t)cfg_.max_grid * cfg_.max_grid * cfg_.max_grid * sizeof(double)) {
        CK(cudaEventSynchronize(ev_nh_));            // the previous admission's upload is done
        std::memcpy(h_nh_, n_H, nhb);
        CK(cudaMemcpyAsync(cells_.nH + c0, h_nh_, nhb, cudaMemcpyHostToDevice, st_));
        CK(cudaEventRecord(ev_nh_, st_));
    } else {
        CK(cudaMemcpyAsync(cells_.nH + c0, n_H, nhb, cudaMemcpyHostToDevice, st_));
        CK(cudaStreamSynchronize(st_));              // n_H is the caller's pageable memory
    }
    CK(launch_init_cells(sims_, s, cells_, proto.ncell, st_));
    flexrt_status r = upload_lists();
    if (r != FLEXRT_OK) return r;
    *slot_out = s;
    return FLEXRT_OK;
}

flexrt_status Engine::add_sources(int s, int32_t n, const int32_t *ijk, const double *ndot) {
    if (s < 0 || s >= (int)slots_.size() || !slots_[s].active) return fail(FLEXRT_E_INVALID, "bad slot");
    if (n < 0 || (n > 0 && (!ijk || !ndot))) return fail(FLEXRT_E_INVALID, "bad source arrays");
    Slot &sl = slots_[s];
    for (int32_t i = 0; i < n; ++i) {
        const int32_t *q = ijk + 3 * i;
        if (q[0] < 0 || q[0] >= sl.h.nx || q[1] < 0 || q[1] >= sl.h.ny || q[2] < 0 || q[2] >= sl.h.nz ||
            !(ndot[i] >= 0.0))
            return fail(FLEXRT_E_INVALID, "source outside the grid or negative rate");
    }
    std::vector<int4> cell = sl.ecell;
    std::vector<double> rate = sl.endot;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t *q = ijk + 3 * i;
        size_t f = cell.size();
        for (size_t k = 0; k < cell.size(); ++k)
            if (cell[k].x == q[0] && cell[k].y == q[1] && cell[k].z == q[2]) { f = k; break; }
        if (f < cell.size()) rate[f] += ndot[i];
        else { cell.push_back(make_int4(q[0], q[1], q[2], s)); rate.push_back(ndot[i]); }
    }
    const int ne = (int)cell.size();
    if (ne > sl.em_n) {
        if (sl.em0 >= 0 && sl.em_n > 0) {
            // grow in place: only the single-simulation engine owns the whole table
            if (slots_.size() != 1 || sl.em0 != 0) return fail(FLEXRT_E_STATE, "sources of a batch member are fixed");
            flexrt_status r = grow_emitters(ne);
            if (r != FLEXRT_OK) return r;
            em_alloc_.reset(em_cap_);
            em_alloc_.alloc(ne);
        } else {
            if (slots_.size() == 1) {
                flexrt_status r = grow_emitters(ne);
                if (r != FLEXRT_OK) return r;
                em_alloc_.reset(em_cap_);
            }
            const long long e0 = em_alloc_.alloc(ne);
            if (e0 < 0) return fail(FLEXRT_E_CAPACITY, "emitter table full");
            sl.em0 = e0;
        }
        sl.em_n = ne;
    }
    sl.ecell = cell;
    sl.endot = rate;
    if (!sl.nref_set && ne > 0) {
        const double mx = *std::max_element(rate.begin(), rate.end());
        if (mx > 0) {
            sl.h.nref = std::ldexp(1.0, (int)std::lround(std::log2(mx * MYR_S * sl.h.inv_ncast)));
            sl.nref_set = true;
            CK(cudaMemcpyAsync((char *)(sims_ + s) + offsetof(SimDev, nref), &sl.h.nref, sizeof(double),
                               cudaMemcpyHostToDevice, st_));
            sl.h.apn_f = atoms_per_nH(sl.h);
            CK(cudaMemcpyAsync((char *)(sims_ + s) + offsetof(SimDev, apn_f), &sl.h.apn_f, sizeof(float),
                               cudaMemcpyHostToDevice, st_));
            if (sl.h.dt > 0) {
                const double dt = sl.h.dt;
                sl.h.dt = 0.0;
                flexrt_status r = set_dt(s, dt);
                if (r != FLEXRT_OK) return r;
                CK(cudaStreamSynchronize(st_));
            }
        }
    }
    std::vector<int32_t> local(ne);
    for (int k = 0; k < ne; ++k) local[k] = k;
    // pageable sources: each copy is staged before the call returns, and
    // runs in stream order behind the steps already enqueued
    CK(cudaMemcpyAsync(em_.cell + sl.em0, cell.data(), ne * sizeof(int4), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(em_.ndot + sl.em0, rate.data(), ne * sizeof(double), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(em_.local + sl.em0, local.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    return upload_lists();
}

flexrt_status Engine::upload_lists() {
    std::vector<int32_t> act;
    std::vector<long long> off;
    std::vector<long long> pref(1, 0), cell0;
    std::vector<int32_t> sim;
    long long run = 0;
    for (int s = 0; s < (int)slots_.size(); ++s) {
        const Slot &sl = slots_[s];
        if (!sl.active) continue;
        const long long ncast = 12LL << (2 * sl.h.l_src);
        for (int k = 0; k < sl.em_n; ++k) {
            act.push_back((int32_t)(sl.em0 + k));
            off.push_back(run);
            run += ncast;
        }
        pref.push_back(pref.back() + sl.h.ncell);
        cell0.push_back(sl.cell0);
        sim.push_back(s);
    }
    if ((long long)act.size() > em_cap_) return fail(FLEXRT_E_CAPACITY, "emitter list");
    // in stream order: the steps already enqueued read the old lists, the
    // next ones the new (pageable sources, staged before each call returns)
    if (!act.empty()) {
        CK(cudaMemcpyAsync(em_.act, act.data(), act.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
        CK(cudaMemcpyAsync(em_.act_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st_));
    }
    if (!sim.empty()) {
        CK(cudaMemcpyAsync(rg_.pref, pref.data(), pref.size() * sizeof(long long), cudaMemcpyHostToDevice, st_));
        CK(cudaMemcpyAsync(rg_.cell0, cell0.data(), cell0.size() * sizeof(long long), cudaMemcpyHostToDevice, st_));
        CK(cudaMemcpyAsync(rg_.sim, sim.data(), sim.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    }
    const long long et = run;
    const int32_t na = (int32_t)act.size(), nr = (int32_t)sim.size();
    const long long nca = pref.back();
    CK(cudaMemcpyAsync((char *)ctl_ + offsetof(Ctl, emit_total), &et, sizeof(et), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync((char *)ctl_ + offsetof(Ctl, n_act_emit), &na, sizeof(na), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync((char *)ctl_ + offsetof(Ctl, n_ranges), &nr, sizeof(nr), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync((char *)ctl_ + offsetof(Ctl, ncell_active), &nca, sizeof(nca), cudaMemcpyHostToDevice, st_));
    return FLEXRT_OK;
}

flexrt_status Engine::set_dt(int s, double dt) {
    if (s < 0 || s >= (int)slots_.size() || !slots_[s].used) return fail(FLEXRT_E_INVALID, "bad slot");
    if (!(dt > 0.0)) return fail(FLEXRT_E_INVALID, "dt must be positive");
    SimDev &h = slots_[s].h;
    if (dt == h.dt) return FLEXRT_OK;
    CK(cudaEventSynchronize(ev_stage_));  // the staging slot's previous upload has been consumed
    h.dt = dt;
    h.gscale = h.nref * h.sigma_ref / (h.dx_phys * h.dx_phys * dt);
    h.hscale = h.gscale * EV_ERG;
    h.dt_f = (float)h.dt; h.gscale_f = (float)h.gscale; h.hscale_f = (float)h.hscale;
    double *st = h_stage_ + 6 * s;
    st[0] = h.dt; st[1] = h.gscale; st[2] = h.hscale;
    float *sf = reinterpret_cast<float *>(st + 3);
    sf[0] = h.dt_f; sf[1] = h.gscale_f; sf[2] = h.hscale_f; sf[3] = 0.0f;
    static_assert(offsetof(SimDev, gscale) == offsetof(SimDev, dt) + sizeof(double), "dt/gscale layout");
    static_assert(offsetof(SimDev, hscale) == offsetof(SimDev, dt) + 2 * sizeof(double), "dt/hscale layout");
    static_assert(offsetof(SimDev, gscale_f) == offsetof(SimDev, dt_f) + sizeof(float), "dt_f layout");
    static_assert(offsetof(SimDev, hscale_f) == offsetof(SimDev, dt_f) + 2 * sizeof(float), "dt_f layout");
    CK(cudaMemcpyAsync((char *)(sims_ + s) + offsetof(SimDev, dt), st, 3 * sizeof(double), cudaMemcpyHostToDevice,
                       st_));
    CK(cudaMemcpyAsync((char *)(sims_ + s) + offsetof(SimDev, dt_f), sf, 3 * sizeof(float), cudaMemcpyHostToDevice,
                       st_));
    CK(cudaEventRecord(ev_stage_, st_));
    return FLEXRT_OK;
}

flexrt_status Engine::poll(bool wait) {
    if (latched_ != FLEXRT_OK) return latched_;
    if (!err_pending_) return FLEXRT_OK;
    if (wait) {
        cudaError_t e = cudaEventSynchronize(ev_err_);
        if (e != cudaSuccess) return cuda(e, "step");
    } else if (cudaEventQuery(ev_err_) != cudaSuccess) {
        return FLEXRT_OK;
    }
    err_pending_ = false;
    static_assert(offsetof(Ctl, par) == 16 && offsetof(Ctl, err) == 20, "ctl layout");
    const int32_t v = h_err_[5];
    q_used_ = reinterpret_cast<const long long *>(h_err_)[h_err_[4] & 1];
    if (v) {
        latched_ = FLEXRT_E_CAPACITY;
        if (v & 1) err_ = "ray queue capacity exceeded; state kept at the last complete step";
        else if (v & 8) err_ = "merge group too heavy for exact weighted sums (more than 2^13 rays as bright as its brightest)";
        else if (v & 2) err_ = "ray older than the rotation ring (internal bound)";
        else err_ = "ray crossed more than four cells in one step (internal bound)";
    }
    return latched_;
}

static cudaEvent_t take_event(std::vector<cudaEvent_t> &pool) {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

flexrt_status Engine::launch_step() {
    flexrt_status r = launch_stage(1);
    return r == FLEXRT_OK ? launch_stage(2) : r;
}

// stage 1: emission and the marches (the trial passes and the committed
// one); stage 2: merge, chemistry and the budget's commit
flexrt_status Engine::launch_stage(int stage) {
    const int ms = (int)slots_.size();
    EmitArgs ea{ctl_, sims_, acc_, {q_[0], q_[1]}, qcap_, em_, pixtab_, ltab_, cfg_.nb};
    MarchArgs ma{ctl_, sims_, acc_, ms, {q_[0], q_[1]}, qcap_, em_, cells_, pixtab_, ltab_, march_slab_};
    ChemArgs ca{ctl_, sims_, acc_, ms, cells_, rg_, 1};
    const bool prof = profiling_ && !cfg_.use_graph;
    cudaEvent_t e0 = nullptr;
    auto tic = [&]() {
        if (prof) { e0 = take_event(ev_pool_); cudaEventRecord(e0, st_); }
    };
    auto toc = [&](int k) {
        if (prof) { cudaEvent_t e1 = take_event(ev_pool_); cudaEventRecord(e1, st_); ev_k_[k].push_back({e0, e1}); }
    };
    if (stage == 1) {
        tic();
        CK(launch_emit(ea, emit_blocks_, st_));
        toc(0);
        // passes of the Gamma - <n_HI> iteration before the committed one: march,
        // trial chemistry (opacity of the time-averaged state), reset of the
        // step's march output and tallies
        int iters = 1;
        for (const Slot &sl : slots_)
            if (sl.used) iters = std::max(iters, (int)sl.h.gamma_iters);
        for (int it = 0; it + 1 < iters; ++it) {
            tic();
            CK(launch_march(ma, cfg_.nb, march_agg_, march_minb_, march_blocks_, march_threads_, st_, ext_variants()));
            toc(1);
            ChemArgs ct = ca;
            ct.final_pass = 0;
            tic();
            CK(launch_chem(ct, chem_blocks_, st_));
            toc(2);
            CK(launch_iter_reset(ctl_, acc_, ms, st_));
    }
        tic();
        CK(launch_march(ma, cfg_.nb, march_agg_, march_minb_, march_blocks_, march_threads_, st_, ext_variants()));
        toc(1);
        return FLEXRT_OK;
    }
    if (merge_built()) {
        MergeArgs ga{ctl_, sims_, acc_, ms, {q_[0], q_[1]}, em_, rg_, pixtab_, ltab_, mw_, cfg_.nb, qcap_};
        tic();
        CK(launch_merge(ga, sm_count_, st_, &mside_));
        toc(3);
    }
    tic();
    CK(launch_chem(ca, chem_blocks_, st_));
    toc(2);
    CK(launch_end(ctl_, sims_, acc_, ms, st_));
    return FLEXRT_OK;
}

void Engine::free_retired() {
    for (auto &sl : slots_) {
        if (sl.used && !sl.active && sl.release_after >= 0 && steps_taken_ > sl.release_after) {
            if (sl.em0 >= 0 && sl.em_n > 0) em_alloc_.release(sl.em0, sl.em_n);
            sl = Slot();
        }
    }
}

flexrt_status Engine::step() {
    if (mid_step_) return fail(FLEXRT_E_STATE, "finish the staged step first");
    flexrt_status s = poll(false);
    if (s != FLEXRT_OK) return s;
    free_retired();
    if (cfg_.use_graph) {
        if (graph_dirty_) {
            if (graph_) { cudaGraphExecDestroy(graph_); graph_ = nullptr; }
            CK(cudaStreamSynchronize(st_));
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
            flexrt_status r = launch_step();
            cudaError_t ee = cudaStreamEndCapture(st_, &g);
            if (r != FLEXRT_OK) { if (g) cudaGraphDestroy(g); return r; }
            if (ee != cudaSuccess) return cuda(ee, "graph capture");
            ee = cudaGraphInstantiate(&graph_, g, 0);
            cudaGraphDestroy(g);
            if (ee != cudaSuccess) return cuda(ee, "graph instantiate");
            graph_dirty_ = false;
        }
        CK(cudaGraphLaunch(graph_, st_));
    } else {
        flexrt_status r = launch_step();
        if (r != FLEXRT_OK) return r;
    }
    // queue counts, parity and error word of the step, read when it completes
    CK(cudaMemcpyAsync(h_err_, ctl_, offsetof(Ctl, err) + sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    CK(cudaEventRecord(ev_err_, st_));
    err_pending_ = true;
    ++steps_taken_;
    for (auto &sl : slots_)
        if (sl.active) ++sl.h.step;
    // the step just enqueued drops the rays of members retired before it;
    // work enqueued later runs after it, so their emitters can be reused
    free_retired();
    return FLEXRT_OK;
}

flexrt_status Engine::step_stage(int stage) {
    if (cfg_.use_graph || slots_.size() != 1) return fail(FLEXRT_E_STATE, "staged steps are for single simulations");
    if (stage == 1) {
        if (mid_step_) return fail(FLEXRT_E_STATE, "a staged step is already open");
        flexrt_status s = poll(false);
        if (s != FLEXRT_OK) return s;
        s = launch_stage(1);
        if (s != FLEXRT_OK) return s;
        mid_step_ = true;
        return FLEXRT_OK;
    }
    if (stage != 2 || !mid_step_) return fail(FLEXRT_E_STATE, "no staged step to finish");
    mid_step_ = false;
    flexrt_status s = launch_stage(2);
    if (s != FLEXRT_OK) return s;
    // queue counts, parity and error word of the step, read when it completes
    CK(cudaMemcpyAsync(h_err_, ctl_, offsetof(Ctl, err) + sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    CK(cudaEventRecord(ev_err_, st_));
    err_pending_ = true;
    ++steps_taken_;
    for (auto &sl : slots_)
        if (sl.active) ++sl.h.step;
    return FLEXRT_OK;
}

flexrt_status Engine::sync() {
    CK(cudaStreamSynchronize(st_));
    return poll(true);
}

flexrt_status Engine::retire(int s) {
    if (s < 0 || s >= (int)slots_.size() || !slots_[s].active) return fail(FLEXRT_E_INVALID, "bad slot");
    Slot &sl = slots_[s];
    sl.active = false;
    sl.h.active = 0;
    const int32_t zero = 0;
    // stream-ordered: the steps already enqueued still advance the member
    CK(cudaMemcpyAsync((char *)(sims_ + s) + offsetof(SimDev, active), &zero, sizeof(zero), cudaMemcpyHostToDevice,
                       st_));
    cell_alloc_.release(sl.cell0, sl.h.ncell);
    sl.release_after = steps_taken_;   // its rays are dropped by the next step's march
    return upload_lists();
}

flexrt_status Engine::reset_all() {
    CK(cudaStreamSynchronize(st_));
    latched_ = FLEXRT_OK;
    err_pending_ = false;
    int32_t derr = 0;
    CK(cudaMemcpy(&derr, &ctl_->err, sizeof(derr), cudaMemcpyDeviceToHost));
    if (derr && mwmem_) {
        // a step that failed may have stopped inside the merge, with groups
        // not cleared: clear the whole merge scratch
        auto it = alloc_sizes_.find(mwmem_);
        if (it != alloc_sizes_.end()) CK(cudaMemset(mwmem_, 0, it->second));
    }
    CK(cudaMemset(ctl_, 0, offsetof(Ctl, emit_total)));   // counts, parity, error
    for (int s = 0; s < (int)slots_.size(); ++s) {
        Slot &sl = slots_[s];
        if (!sl.active) continue;
        sl.h.step = 0;
        const int32_t zero = 0;
        CK(cudaMemcpy((char *)(sims_ + s) + offsetof(SimDev, step), &zero, sizeof(zero), cudaMemcpyHostToDevice));
        // keep the monotonic marched-ray counter (last field) for profiling windows
        CK(cudaMemset(acc_ + s, 0, offsetof(SimAcc, rays_in_total)));
        CK(launch_init_cells(sims_, s, cells_, sl.h.ncell, st_));
    }
    CK(cudaStreamSynchronize(st_));
    return FLEXRT_OK;
}

flexrt_status Engine::read_acc(int s, SimAcc &a) {
    CK(cudaStreamSynchronize(st_));
    CK(cudaMemcpy(&a, acc_ + s, sizeof(a), cudaMemcpyDeviceToHost));
    return FLEXRT_OK;
}

// Runs fn(i0, i1) over [0, n) on up to eight host threads (one when n is
// small): the read-back's conversions write the caller's arrays in parallel.
template <typename F>
static void host_parallel(size_t n, F fn) {
    const size_t nt = n >= (1u << 20) ? 8 : 1;
    if (nt == 1) { fn((size_t)0, n); return; }
    std::vector<std::thread> th;
    const size_t per = (n + nt - 1) / nt;
    for (size_t k = 1; k < nt; ++k) {
        const size_t i0 = std::min(n, k * per), i1 = std::min(n, (k + 1) * per);
        th.emplace_back([=]() { fn(i0, i1); });
    }
    fn((size_t)0, std::min(n, per));
    for (auto &t : th) t.join();
}

flexrt_status Engine::fields(int s, flexrt_fields *f) {
    const Slot *sl = slot(s);
    if (!sl || !f) return fail(FLEXRT_E_INVALID, "bad slot or fields");
    const size_t n = (size_t)sl->h.ncell;
    const long long c0 = sl->cell0;
    // the cells' words go to pinned staging in stream order (neutral
    // fraction, n_H, then the single-precision x, T, Gamma), then the host
    // converts them into the caller's double arrays
    const size_t need = n * (2 * sizeof(double) + 3 * sizeof(float));
    if (need > h_fields_bytes_) {
        if (h_fields_) { CK(cudaStreamSynchronize(st_)); cudaFreeHost(h_fields_); h_fields_ = nullptr; h_fields_bytes_ = 0; }
        if (cudaMallocHost(&h_fields_, need) != cudaSuccess) return fail(FLEXRT_E_OOM, "pinned allocation failed");
        h_fields_bytes_ = need;
    }
    double *hy = static_cast<double *>(h_fields_), *hn = hy + n;
    float *hx = reinterpret_cast<float *>(hn + n), *hT = hx + n, *hg = hT + n;
    if (f->n_HI) {
        CK(cudaMemcpyAsync(hy, cells_.y + c0, n * sizeof(double), cudaMemcpyDeviceToHost, st_));
        CK(cudaMemcpyAsync(hn, cells_.nH + c0, n * sizeof(double), cudaMemcpyDeviceToHost, st_));
    }
    if (f->x_HII) CK(cudaMemcpyAsync(hx, cells_.x + c0, n * sizeof(float), cudaMemcpyDeviceToHost, st_));
    if (f->T) CK(cudaMemcpyAsync(hT, cells_.T + c0, n * sizeof(float), cudaMemcpyDeviceToHost, st_));
    if (f->gamma_HI) CK(cudaMemcpyAsync(hg, cells_.gamma + c0, n * sizeof(float), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    poll(true);                                   // latch a failed step's error (the state is kept)
    host_parallel(n, [&](size_t i0, size_t i1) {
        if (f->n_HI)
            for (size_t i = i0; i < i1; ++i) f->n_HI[i] = hn[i] * hy[i];
        if (f->x_HII)
            for (size_t i = i0; i < i1; ++i) f->x_HII[i] = hx[i];
        if (f->T)
            for (size_t i = i0; i < i1; ++i) f->T[i] = hT[i];
        if (f->gamma_HI)
            for (size_t i = i0; i < i1; ++i) f->gamma_HI[i] = hg[i];
    });
    return FLEXRT_OK;
}

flexrt_status Engine::budget(int s, double out[4]) {
    const Slot *sl = slot(s);
    if (!sl || !out) return fail(FLEXRT_E_INVALID, "bad slot");
    SimAcc a;
    flexrt_status r = read_acc(s, a);
    if (r != FLEXRT_OK) return r;
    const double k = sl->h.nref;
    out[0] = a.emitted * k; out[1] = a.absorbed * k; out[2] = a.escaped * k; out[3] = a.in_flight * k;
    return FLEXRT_OK;
}

flexrt_status Engine::screen_excess(int s, double *out) {
    const Slot *sl = slot(s);
    if (!sl || !out) return fail(FLEXRT_E_INVALID, "bad slot");
    SimAcc a;
    flexrt_status r = read_acc(s, a);
    if (r != FLEXRT_OK) return r;
    *out = a.lost * sl->h.nref;
    return FLEXRT_OK;
}

flexrt_status Engine::counts(int s, int64_t out[6]) {
    const Slot *sl = slot(s);
    if (!sl || !out) return fail(FLEXRT_E_INVALID, "bad slot");
    SimAcc a;
    flexrt_status r = read_acc(s, a);
    if (r != FLEXRT_OK) return r;
    int32_t step = 0;
    CK(cudaMemcpy(&step, (char *)(sims_ + s) + offsetof(SimDev, step), sizeof(step), cudaMemcpyDeviceToHost));
    out[0] = (int64_t)a.rays_live; out[1] = (int64_t)a.seg_last; out[2] = (int64_t)a.seg_total;
    out[3] = step; out[4] = cfg_.ray_capacity; out[5] = (int64_t)a.rays_in_last;
    return FLEXRT_OK;
}

flexrt_status Engine::segment_counts(int s, int32_t *out) {
    const Slot *sl = slot(s);
    if (!sl || !out) return fail(FLEXRT_E_INVALID, "bad slot");
    if (!cells_.segcnt) return fail(FLEXRT_E_STATE, "created without keep_diagnostics");
    CK(cudaStreamSynchronize(st_));
    CK(cudaMemcpy(out, cells_.segcnt + sl->cell0, (size_t)sl->h.ncell * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return FLEXRT_OK;
}

// the live rays of simulation s in queue order: indices into the queue copy
static std::vector<long long> member_rays(const std::vector<uint32_t> &pl, const std::vector<uint32_t> &em,
                                          const std::vector<uint32_t> &ma, int s, long long em0, int em_n) {
    std::vector<long long> idx;
    for (long long i = 0; i < (long long)pl.size(); ++i) {
        if (pl[i] == DEAD_RAY) continue;
        if (em[i] & MERGED_BIT) {
            if (ma.empty() || (int)((ma[i] >> 16) & 0x7fffu) != s) continue;
        } else if ((long long)em[i] < em0 || (long long)em[i] >= em0 + em_n) {
            continue;
        }
        idx.push_back(i);
    }
    return idx;
}

flexrt_status Engine::rays(int s, int64_t cap, int32_t *level, int64_t *pixel, int32_t *emitter, int32_t *birth,
                           int32_t *dir, double *photons, int64_t *n) {
    const Slot *sl = slot(s);
    if (!sl || !n || cap < 0) return fail(FLEXRT_E_INVALID, "bad arguments");
    SimAcc a;
    flexrt_status r = read_acc(s, a);
    if (r != FLEXRT_OK) return r;
    *n = (int64_t)a.rays_live;
    Ctl hc;
    CK(cudaMemcpy(&hc, ctl_, sizeof(hc), cudaMemcpyDeviceToHost));
    const int qs = mid_step_ ? hc.par ^ 1 : hc.par;     // between the stages: the march's output
    const long long m = hc.cnt[qs];
    if (mid_step_) *n = 0;
    if (m == 0 || cap == 0) {
        if (mid_step_ && m > 0) {
            std::vector<uint32_t> pl(m), em(m), ma(merge_built() ? m : 0);
            CK(cudaMemcpy(pl.data(), q_[qs].pl, m * 4, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(em.data(), q_[qs].em, m * 4, cudaMemcpyDeviceToHost));
            if (!ma.empty()) CK(cudaMemcpy(ma.data(), q_[qs].ma, m * 4, cudaMemcpyDeviceToHost));
            *n = (int64_t)member_rays(pl, em, ma, s, sl->em0, sl->em_n).size();
        }
        return FLEXRT_OK;
    }
    const Queue &q = q_[qs];
    std::vector<uint32_t> pl(m), em(m), ma(merge_built() ? m : 0);
    std::vector<int32_t> bi(m), d(3 * m);
    CK(cudaMemcpy(pl.data(), q.pl, m * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(em.data(), q.em, m * 4, cudaMemcpyDeviceToHost));
    if (!ma.empty()) CK(cudaMemcpy(ma.data(), q.ma, m * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bi.data(), q.bi, m * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(d.data(), q.dx, m * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(d.data() + m, q.dy, m * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(d.data() + 2 * m, q.dz, m * 4, cudaMemcpyDeviceToHost));
    std::vector<std::vector<float>> ph(photons ? sl->h.nb : 0, std::vector<float>(m));
    for (int b = 0; b < (int)ph.size(); ++b) CK(cudaMemcpy(ph[b].data(), q.ph[b], m * 4, cudaMemcpyDeviceToHost));
    const std::vector<long long> idx = member_rays(pl, em, ma, s, sl->em0, sl->em_n);
    if (mid_step_) *n = (int64_t)idx.size();
    for (long long k = 0; k < (long long)idx.size() && k < cap; ++k) {
        const long long i = idx[k];
        if (level) level[k] = (int32_t)(pl[i] >> LEVEL_SHIFT);
        if (pixel) pixel[k] = (int64_t)(pl[i] & PIX_MASK);
        if (emitter)
            emitter[k] = (em[i] & MERGED_BIT) ? -1 - (int32_t)(em[i] & ~MERGED_BIT) : (int32_t)(em[i] - sl->em0);
        if (birth) birth[k] = bi[i];
        if (dir) { dir[3 * k] = d[i]; dir[3 * k + 1] = d[m + i]; dir[3 * k + 2] = d[2 * m + i]; }
        for (int b = 0; b < (int)ph.size(); ++b) photons[(size_t)sl->h.nb * k + b] = (double)ph[b][i] * sl->h.nref;
    }
    return FLEXRT_OK;
}

flexrt_status Engine::rays_merged(int s, int64_t cap, int32_t *merged, int32_t *vertex, int32_t *dist, int64_t *pos,
                                  double *thr, int64_t *n) {
    const Slot *sl = slot(s);
    if (!sl || !n || cap < 0) return fail(FLEXRT_E_INVALID, "bad arguments");
    CK(cudaStreamSynchronize(st_));
    Ctl hc;
    CK(cudaMemcpy(&hc, ctl_, sizeof(hc), cudaMemcpyDeviceToHost));
    const int qs = mid_step_ ? hc.par ^ 1 : hc.par;
    const long long m = hc.cnt[qs];
    const Queue &q = q_[qs];
    std::vector<uint32_t> pl(m), em(m), ma(merge_built() ? m : 0);
    std::vector<int32_t> mx(ma.size()), my(ma.size()), mz(ma.size());
    std::vector<float> mt(ma.size());
    if (m > 0) {
        CK(cudaMemcpy(pl.data(), q.pl, m * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(em.data(), q.em, m * 4, cudaMemcpyDeviceToHost));
    }
    if (!ma.empty()) {
        CK(cudaMemcpy(ma.data(), q.ma, m * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(mx.data(), q.mx, m * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(my.data(), q.my, m * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(mz.data(), q.mz, m * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(mt.data(), q.mthr, m * 4, cudaMemcpyDeviceToHost));
    }
    const std::vector<long long> idx = member_rays(pl, em, ma, s, sl->em0, sl->em_n);
    *n = (int64_t)idx.size();
    for (long long k = 0; k < (long long)idx.size() && k < cap; ++k) {
        const long long i = idx[k];
        const bool mg = (em[i] & MERGED_BIT) != 0;
        if (merged) merged[k] = mg ? 1 : 0;
        if (vertex) vertex[k] = mg && (ma[i] >> 31) ? 1 : 0;
        if (dist) dist[k] = mg ? (int32_t)(ma[i] & 0xffffu) : 0;
        if (pos) {
            pos[3 * k] = mg ? mx[i] : 0; pos[3 * k + 1] = mg ? my[i] : 0; pos[3 * k + 2] = mg ? mz[i] : 0;
        }
        if (thr) thr[k] = mg ? (double)mt[i] * sl->h.nref : 0.0;
    }
    return FLEXRT_OK;
}

flexrt_status Engine::ionized_volume(int s, double *x_ion) {
    const Slot *sl = slot(s);
    if (!sl || !x_ion) return fail(FLEXRT_E_INVALID, "bad slot or buffer");
    CK(cudaStreamSynchronize(st_));
    poll(true);
    std::vector<double> v((size_t)sl->h.ncell);
    CK(cudaMemcpy(v.data(), cells_.xion + sl->cell0, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < v.size(); ++i) x_ion[i] = sl->h.gen_mode ? (double)v[i] : 0.0;
    return FLEXRT_OK;
}

flexrt_status Engine::set_launch(int agg, int minb, int blocks_per_sm, int threads, int slab) {
    if (threads == 0) threads = 256;
    if (slab == 0) slab = OUT_SLAB;
    if (!march_variant_exists(cfg_.nb, agg, minb, ext_variants()) || blocks_per_sm < 0 || blocks_per_sm > 32 ||
        (threads != 128 && threads != 256) || slab < 32 || slab > 4096)
        return fail(FLEXRT_E_INVALID, "march kernel variant not built or launch shape out of range");
    CK(march_prepare(cfg_.nb, agg, minb, (int)slots_.size(), ext_variants()));
    const int lim = march_max_blocks_per_sm(cfg_.nb, agg, minb, threads, (int)slots_.size(), ext_variants());
    if (lim < 1) return fail(FLEXRT_E_INVALID, "variant cannot be resident");
    const int bps = blocks_per_sm == 0 ? lim : std::min(blocks_per_sm, lim);
    march_agg_ = agg;
    march_minb_ = minb;
    march_threads_ = threads;
    march_slab_ = slab;
    march_blocks_ = sm_count_ * bps;
    graph_dirty_ = true;
    return FLEXRT_OK;
}

flexrt_status Engine::profile(bool on) {
    double ms[4];
    int64_t l[4], r = 0;
    flexrt_status s = kernel_times(ms, l, &r);
    profiling_ = on;
    return s;
}

flexrt_status Engine::kernel_times(double ms[4], int64_t launches[4], int64_t *rays) {
    CK(cudaStreamSynchronize(st_));
    for (int k = 0; k < 4; ++k) {
        double t = 0.0;
        for (auto &p : ev_k_[k]) {
            float x = 0.f;
            cudaEventElapsedTime(&x, p.first, p.second);
            t += x;
            ev_pool_.push_back(p.first);
            ev_pool_.push_back(p.second);
        }
        ms[k] = t;
        launches[k] = (int64_t)ev_k_[k].size();
        ev_k_[k].clear();
    }
    std::vector<SimAcc> a(slots_.size());
    CK(cudaMemcpy(a.data(), acc_, a.size() * sizeof(SimAcc), cudaMemcpyDeviceToHost));
    double tot = 0.0;
    for (auto &x : a) tot += x.rays_in_total;
    if (rays) *rays = (int64_t)(tot - rays_at_profile_);
    rays_at_profile_ = tot;
    return FLEXRT_OK;
}

int Engine::free_slots() const {
    int n = 0;
    for (auto &s : slots_) n += s.used ? 0 : 1;
    return n;
}

flexrt_status Engine::queue_used(long long *n) {
    // the count after the last step seen complete (without waiting for the
    // GPU); exact after sync()
    flexrt_status r = poll(false);
    *n = q_used_;
    return r;
}

int Engine::active_count() const {
    int n = 0;
    for (auto &s : slots_) n += s.active ? 1 : 0;
    return n;
}

// ---------------------------------------------------------------------------
// Checkpoint of a single-simulation engine: everything a later step reads --
// the per-cell state, the live ray queue, the emitters' per-step photons and
// rotation ring, the step counter, dt and the photon budget.  Buffers that
// are zero between steps (deposits, screen tallies, merge groups) are not
// stored.  Layout: a header, then the arrays in a fixed order.
// ---------------------------------------------------------------------------
namespace {
struct StateHeader {
    char magic[8];
    int32_t version, nx, ny, nz, nb, n_emitters, ring_w, merged_fields;
    int64_t ncell, nray, step;
    double dt, nref;
    int64_t bytes;
};
constexpr char STATE_MAGIC[8] = {'F', 'L', 'E', 'X', 'R', 'T', 'S', '1'};
}  // namespace

flexrt_status Engine::save_state(int s, void *buf, int64_t cap, int64_t *bytes) {
    const Slot *sl = slot(s);
    if (!sl || !bytes || slots_.size() != 1) return fail(FLEXRT_E_INVALID, "checkpoints are for single simulations");
    if (mid_step_) return fail(FLEXRT_E_STATE, "finish the staged step first");
    CK(cudaStreamSynchronize(st_));
    flexrt_status ps = poll(true);
    if (ps != FLEXRT_OK) return ps;
    Ctl hc;
    CK(cudaMemcpy(&hc, ctl_, sizeof(hc), cudaMemcpyDeviceToHost));
    const long long nray = hc.cnt[hc.par], nc = sl->h.ncell, ne = sl->em_n, rw = em_.ring_w;
    const int nb = cfg_.nb;
    const bool mf = merge_built();
    // (device pointer, bytes) in file order
    std::vector<std::pair<const void *, size_t>> parts = {
        {acc_ + s, sizeof(SimAcc)},
        {cells_.y + sl->cell0, nc * 8}, {cells_.x + sl->cell0, nc * 4}, {cells_.T + sl->cell0, nc * 4},
        {cells_.gamma + sl->cell0, nc * 4}, {cells_.kap + sl->cell0, nc * 8}, {cells_.xion + sl->cell0, nc * 8},
        {cells_.rho + sl->cell0, nc * 4},
        {em_.n0 + sl->em0, (size_t)ne * 4}, {em_.ring + sl->em0 * rw * 3, (size_t)ne * rw * 3 * sizeof(int4)}};
    if (ne == 0) { parts[8].second = 0; parts[9].second = 0; }
    const Queue &q = q_[hc.par];
    const void *qa[] = {q.pl, q.em, q.bi, q.dx, q.dy, q.dz};
    for (const void *a : qa) parts.push_back({a, (size_t)nray * 4});
    for (int b = 0; b < nb; ++b) parts.push_back({q.ph[b], (size_t)nray * 4});
    if (mf) {
        const void *ma[] = {q.mx, q.my, q.mz, q.ma, q.mthr};
        for (const void *a : ma) parts.push_back({a, (size_t)nray * 4});
    }
    size_t tot = sizeof(StateHeader);
    for (auto &p : parts) tot += p.second;
    *bytes = (int64_t)tot;
    if (!buf) return FLEXRT_OK;
    if (cap < (int64_t)tot) return fail(FLEXRT_E_CAPACITY, "checkpoint buffer too small");
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, STATE_MAGIC, 8);
    h.version = 1;
    h.nx = sl->h.nx; h.ny = sl->h.ny; h.nz = sl->h.nz; h.nb = nb;
    h.n_emitters = sl->em_n; h.ring_w = (int32_t)rw; h.merged_fields = mf ? 1 : 0;
    h.ncell = nc; h.nray = nray; h.step = sl->h.step; h.dt = sl->h.dt; h.nref = sl->h.nref;
    h.bytes = (int64_t)tot;
    char *o = (char *)buf;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (auto &p : parts) {
        if (p.second) CK(cudaMemcpy(o, p.first, p.second, cudaMemcpyDeviceToHost));
        o += p.second;
    }
    return FLEXRT_OK;
}

flexrt_status Engine::load_state(int s, const void *buf, int64_t bytes) {
    Slot *sl = (s >= 0 && s < (int)slots_.size() && slots_[s].used) ? &slots_[s] : nullptr;
    if (!sl || !buf || slots_.size() != 1) return fail(FLEXRT_E_INVALID, "checkpoints are for single simulations");
    if (mid_step_) return fail(FLEXRT_E_STATE, "finish the staged step first");
    StateHeader h;
    if (bytes < (int64_t)sizeof(h)) return fail(FLEXRT_E_INVALID, "checkpoint truncated");
    std::memcpy(&h, buf, sizeof(h));
    const int nb = cfg_.nb;
    const long long nc = sl->h.ncell, ne = sl->em_n, rw = em_.ring_w;
    if (std::memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.version != 1 || h.bytes != bytes)
        return fail(FLEXRT_E_INVALID, "not a checkpoint of this library");
    if (h.nx != sl->h.nx || h.ny != sl->h.ny || h.nz != sl->h.nz || h.nb != nb || h.n_emitters != ne ||
        h.ring_w != rw || h.merged_fields != (merge_built() ? 1 : 0) || h.ncell != nc || h.nref != sl->h.nref)
        return fail(FLEXRT_E_INVALID, "checkpoint of a different simulation (grid, bins, sources or layout)");
    if (h.nray < 0 || h.nray > cfg_.ray_capacity) return fail(FLEXRT_E_CAPACITY, "checkpoint holds more rays than the queue");
    const long long nray = h.nray;
    std::vector<std::pair<void *, size_t>> parts = {
        {acc_ + s, sizeof(SimAcc)},
        {cells_.y + sl->cell0, nc * 8}, {cells_.x + sl->cell0, nc * 4}, {cells_.T + sl->cell0, nc * 4},
        {cells_.gamma + sl->cell0, nc * 4}, {cells_.kap + sl->cell0, nc * 8}, {cells_.xion + sl->cell0, nc * 8},
        {cells_.rho + sl->cell0, nc * 4},
        {em_.n0 + sl->em0, (size_t)ne * 4}, {em_.ring + sl->em0 * rw * 3, (size_t)ne * rw * 3 * sizeof(int4)}};
    if (ne == 0) { parts[8].second = 0; parts[9].second = 0; }
    const Queue &q = q_[0];
    void *qa[] = {q.pl, q.em, q.bi, q.dx, q.dy, q.dz};
    for (void *a : qa) parts.push_back({a, (size_t)nray * 4});
    for (int b = 0; b < nb; ++b) parts.push_back({q.ph[b], (size_t)nray * 4});
    if (merge_built()) {
        void *ma[] = {q.mx, q.my, q.mz, q.ma, q.mthr};
        for (void *a : ma) parts.push_back({a, (size_t)nray * 4});
    }
    size_t tot = sizeof(StateHeader);
    for (auto &p : parts) tot += p.second;
    if ((int64_t)tot != bytes) return fail(FLEXRT_E_INVALID, "checkpoint size does not match its header");
    CK(cudaStreamSynchronize(st_));
    const char *src = (const char *)buf + sizeof(h);
    for (auto &p : parts) {
        if (p.second) CK(cudaMemcpy(p.first, src, p.second, cudaMemcpyHostToDevice));
        src += p.second;
    }
    // the live rays in queue 0, nothing in flight in queue 1, no latched error
    const long long cnt[2] = {nray, 0};
    const int32_t par_err[2] = {0, 0};
    static_assert(offsetof(Ctl, err) == offsetof(Ctl, par) + sizeof(int32_t), "ctl layout");
    CK(cudaMemcpy(ctl_->cnt, cnt, sizeof(cnt), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&ctl_->par, par_err, sizeof(par_err), cudaMemcpyHostToDevice));
    sl->h.step = (int32_t)h.step;
    CK(cudaMemcpy((char *)(sims_ + s) + offsetof(SimDev, step), &sl->h.step, sizeof(int32_t), cudaMemcpyHostToDevice));
    latched_ = FLEXRT_OK;
    err_pending_ = false;
    if (h.dt > 0.0) {
        flexrt_status r = set_dt(s, h.dt);
        if (r != FLEXRT_OK) return r;
    }
    CK(cudaStreamSynchronize(st_));
    return FLEXRT_OK;
}

}  // namespace frt
