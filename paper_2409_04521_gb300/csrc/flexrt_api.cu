// flexrt_api.cu -- host engine and the C ABI declared in include/flexrt.h.
//
// One flexrt_ctx owns one simulation: its cells, emitters and the double-
// buffered structure-of-arrays ray queue, all in device memory.  A step is
// four launches on the context stream (emit, march, chem, end); every size
// the kernels need is read from device memory.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/flexrt.h"
#include "frt_launch.h"

using namespace frt;

namespace {

constexpr double EV_ERG = 1.602176634e-12;
constexpr double MYR_S = 3.15576e13;

// process-wide fixed-point pixel vector tables, one per device, grown on demand
struct PixTable {
    int4 *ptr = nullptr;
    int level = -1;
};
std::mutex g_tab_mu;
std::map<int, PixTable> g_tabs;

cudaError_t get_pixtab(int device, int level, cudaStream_t st, const int4 **out) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    PixTable &t = g_tabs[device];
    if (t.level < level) {
        int4 *p = nullptr;
        size_t bytes = (size_t)(4LL * ((1LL << (2 * (level + 1))) - 1)) * sizeof(int4);
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

void split_table(double nmin, int32_t *K) {
    double f = std::sqrt(3.0 / (M_PI * nmin));
    for (int l = 0; l < 16; ++l) {
        double r = std::ldexp(f, l);
        long long k = (long long)std::ceil(r);
        if (k < 1) k = 1;
        if (k > (1LL << 30)) k = 1LL << 30;
        K[l] = (int32_t)k;
    }
}

}  // namespace

struct flexrt_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nb = 1;
    long long cap = 0;
    long long ncell = 0;
    std::string err;
    flexrt_status latched = FLEXRT_OK;

    Ctl *ctl = nullptr;
    SimDev *sims = nullptr;
    SimAcc *acc = nullptr;
    void *qmem = nullptr;
    Queue q[2];
    Cells cells{};
    Emitters em{};
    Ranges rg{};
    const int4 *pixtab = nullptr;
    int ltab = 0;
    int march_blocks = 0, march_threads = 256, chem_blocks = 0;
    int march_agg = 0, march_minb = 3, sm_count = 1;

    SimDev h{};  // host copy of the simulation constants
    int ecap = 0;
    std::vector<int4> hcell;
    std::vector<double> hndot;
    bool nref_set = false;

    // pinned staging
    int32_t *h_err = nullptr;
    double *h_dt = nullptr;
    cudaEvent_t ev_err = nullptr, ev_dt = nullptr;
    bool err_pending = false;

    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_k[3];
    double rays_total_at_profile = 0.0;

    flexrt_status fail(flexrt_status s, const std::string &m) {
        err = m;
        return s;
    }
    flexrt_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return FLEXRT_OK;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return FLEXRT_E_CUDA;
    }
};

#define CK(ctx, call)                                                 \
    do {                                                              \
        cudaError_t e__ = (call);                                     \
        if (e__ != cudaSuccess) return (ctx)->cuda(e__, #call);       \
    } while (0)

static void free_ctx(flexrt_ctx *c) {
    if (!c) return;
    cudaFree(c->ctl); cudaFree(c->sims); cudaFree(c->acc); cudaFree(c->qmem);
    cudaFree(c->cells.nH); cudaFree(c->cells.y); cudaFree(c->cells.x); cudaFree(c->cells.T); cudaFree(c->cells.gamma);
    cudaFree(c->cells.kap); cudaFree(c->cells.dep); cudaFree(c->cells.segcnt);
    cudaFree(c->em.cell); cudaFree(c->em.local); cudaFree(c->em.ndot); cudaFree(c->em.n0);
    cudaFree(c->em.ring); cudaFree(c->em.act); cudaFree(c->em.act_off);
    cudaFree(c->rg.pref); cudaFree(c->rg.cell0); cudaFree(c->rg.sim);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_dt) cudaFreeHost(c->h_dt);
    if (c->ev_err) cudaEventDestroy(c->ev_err);
    if (c->ev_dt) cudaEventDestroy(c->ev_dt);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto &v : c->ev_k)
        for (auto &p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

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

static size_t ray_bytes(int nb) { return 6 * sizeof(int32_t) + (size_t)nb * sizeof(float); }

static cudaError_t alloc_queue(flexrt_ctx *c) {
    size_t per = ray_bytes(c->nb);
    size_t bytes = per * (size_t)c->cap;
    char *base = nullptr;
    cudaError_t e = cudaMalloc(&base, 2 * bytes + 256);
    if (e != cudaSuccess) return e;
    c->qmem = base;
    for (int k = 0; k < 2; ++k) {
        char *p = base + k * bytes;
        size_t a = (size_t)c->cap * 4;
        c->q[k].pl = (uint32_t *)p; p += a;
        c->q[k].em = (uint32_t *)p; p += a;
        c->q[k].bi = (int32_t *)p; p += a;
        c->q[k].dx = (int32_t *)p; p += a;
        c->q[k].dy = (int32_t *)p; p += a;
        c->q[k].dz = (int32_t *)p; p += a;
        for (int b = 0; b < MAXB; ++b) {
            c->q[k].ph[b] = b < c->nb ? (float *)p : nullptr;
            if (b < c->nb) p += a;
        }
    }
    return cudaSuccess;
}

extern "C" flexrt_status flexrt_create(const flexrt_grid *grid, const flexrt_box *box, const double *n_H,
                                       const flexrt_mfp *mfp, const flexrt_spectrum *sp,
                                       const flexrt_options *opt_in, flexrt_ctx **out) {
    if (!out) return FLEXRT_E_INVALID;
    *out = nullptr;
    if (!grid || !box || !n_H || !sp) return FLEXRT_E_INVALID;
    flexrt_options opt;
    if (opt_in) opt = *opt_in; else flexrt_default_options(&opt);
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nx > 1000 || grid->ny > 1000 || grid->nz > 1000)
        return FLEXRT_E_INVALID;
    if (sp->nbins < 1 || sp->nbins > FLEXRT_MAX_BINS || !sp->frac || !sp->sigma_cm2 || !sp->eheat_erg)
        return FLEXRT_E_INVALID;
    if (opt.l_src < 0 || opt.l_max < opt.l_src || opt.l_max > FLEXRT_MAX_LEVEL || !(opt.n_ray_min > 0) ||
        opt.chem_iters < 1 || !(box->box_cm_comoving > 0) || box->redshift <= -1.0)
        return FLEXRT_E_INVALID;

    flexrt_ctx *c = new (std::nothrow) flexrt_ctx();
    if (!c) return FLEXRT_E_OOM;
    auto bail = [&](flexrt_status s) { free_ctx(c); return s; };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(FLEXRT_E_CUDA);
    if (opt.cuda_stream) c->st = (cudaStream_t)opt.cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) return bail(FLEXRT_E_CUDA);
        c->own_stream = true;
    }
    c->nb = sp->nbins;
    c->ncell = (long long)grid->nx * grid->ny * grid->nz;

    // simulation constants
    SimDev &h = c->h;
    std::memset(&h, 0, sizeof(h));
    h.nx = grid->nx; h.ny = grid->ny; h.nz = grid->nz; h.nb = sp->nbins;
    h.cell_off = 0; h.ncell = c->ncell;
    h.l_src = opt.l_src; h.l_max = opt.l_max;
    split_table(opt.n_ray_min, h.K);
    h.active = 1; h.step = 0;
    double diag = std::sqrt((double)grid->nx * grid->nx + (double)grid->ny * grid->ny + (double)grid->nz * grid->nz);
    h.ring_w = (int)std::ceil(diag) + 4;
    h.rotate = opt.rotate ? 1 : 0;
    h.seed = opt.seed;
    h.eps_term = (float)opt.eps_term;
    h.sigma_ref = sp->sigma_cm2[0];
    if (!(h.sigma_ref > 0)) return bail(FLEXRT_E_INVALID);
    for (int b = 0; b < sp->nbins; ++b) {
        h.sig[b] = (float)(sp->sigma_cm2[b] / h.sigma_ref);
        h.sige[b] = (float)(sp->sigma_cm2[b] / h.sigma_ref * sp->eheat_erg[b] / EV_ERG);
        h.frac[b] = (float)sp->frac[b];
    }
    h.dt = 0.0; h.gscale = 0.0;
    h.dx_com = box->box_cm_comoving / grid->nx;
    h.dx_phys = h.dx_com / (1.0 + box->redshift);
    h.inv_ncast = 1.0 / (double)(12LL << (2 * opt.l_src));
    h.z = box->redshift;
    {
        const double kB = 1.380649e-16, sT = 6.6524587e-25, a = 7.5657e-15, me = 9.1093837e-28, cl = 2.99792458e10;
        double Tc = 2.7255 * (1.0 + box->redshift);
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
    if ((m.mode == 1 || m.mode == 2) && !(m.lambda0_cm_comoving > 0)) return bail(FLEXRT_E_INVALID);
    if (m.mode == 2 && !(m.gamma_ref > 0)) return bail(FLEXRT_E_INVALID);
    double mean = m.nH_mean;
    if (!(mean > 0)) {
        double s = 0.0;
        for (long long i = 0; i < c->ncell; ++i) s += n_H[i];
        mean = s / (double)c->ncell;
    }
    h.nH_mean = mean;
    h.ksc = h.sigma_ref * h.dx_phys;
    h.inv_nH_mean = 1.0 / mean;
    h.inv_gamma_ref = m.gamma_ref > 0 ? 1.0 / m.gamma_ref : 0.0;
    h.y_thr = 1.0 - m.xion_threshold;
    h.kap_sub0 = m.lambda0_cm_comoving > 0 ? (float)(h.dx_com / m.lambda0_cm_comoving) : 0.0f;
    h.x_init = opt.x_init; h.T_init = opt.T_init;
    h.nref = 1.0;

    // pixel table level: deepest level a ray can reach before leaving the box
    int L = h.l_src;
    while (L < h.l_max && h.K[L] <= h.ring_w) ++L;
    c->ltab = std::min(L, 11);

    // queue capacity
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    long long cap = opt.ray_capacity;
    if (cap <= 0) cap = (long long)(0.3 * (double)freeb / (2.0 * ray_bytes(c->nb)));
    cap = std::max(cap, 1024LL);
    c->cap = cap;

    if (alloc_queue(c) != cudaSuccess) return bail(FLEXRT_E_OOM);
#define ALLOC(ptr, n) \
    if (cudaMalloc(&(ptr), (size_t)(n) * sizeof(*(ptr))) != cudaSuccess) return bail(FLEXRT_E_OOM)
    ALLOC(c->ctl, 1);
    ALLOC(c->sims, 1);
    ALLOC(c->acc, 1);
    ALLOC(c->cells.nH, c->ncell);
    ALLOC(c->cells.y, c->ncell);
    ALLOC(c->cells.x, c->ncell);
    ALLOC(c->cells.T, c->ncell);
    ALLOC(c->cells.gamma, c->ncell);
    ALLOC(c->cells.kap, c->ncell);
    ALLOC(c->cells.dep, c->ncell);
    if (opt.keep_diagnostics) ALLOC(c->cells.segcnt, c->ncell);
    ALLOC(c->rg.pref, 2);
    ALLOC(c->rg.cell0, 1);
    ALLOC(c->rg.sim, 1);
#undef ALLOC
    if (cudaMallocHost(&c->h_err, 64) != cudaSuccess) return bail(FLEXRT_E_OOM);
    if (cudaMallocHost(&c->h_dt, 64) != cudaSuccess) return bail(FLEXRT_E_OOM);
    cudaEventCreateWithFlags(&c->ev_err, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_dt, cudaEventDisableTiming);
    c->em.ring_w = h.ring_w;

    e = get_pixtab(c->device, c->ltab, c->st, &c->pixtab);
    if (e != cudaSuccess) { c->cuda(e, "pixel table"); return bail(FLEXRT_E_CUDA); }

    Ctl hc{};
    hc.n_ranges = 1;
    hc.ncell_active = c->ncell;
    long long pref[2] = {0, c->ncell};
    long long cell0 = 0;
    int32_t s0 = 0;
    if (cudaMemcpyAsync(c->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->sims, &h, sizeof(h), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemsetAsync(c->acc, 0, sizeof(SimAcc), c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->rg.pref, pref, sizeof(pref), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->rg.cell0, &cell0, sizeof(cell0), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->rg.sim, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->cells.nH, n_H, (size_t)c->ncell * sizeof(double), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess)
        return bail(FLEXRT_E_CUDA);
    if (launch_init_cells(c->sims, 0, c->cells, c->ncell, c->st) != cudaSuccess) return bail(FLEXRT_E_CUDA);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return bail(FLEXRT_E_CUDA);

    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    c->sm_count = std::max(dev_sms, 1);
    if (!march_variant_exists(c->nb, c->march_agg, c->march_minb)) { c->march_agg = 0; c->march_minb = 2; }
    int per_sm = march_max_blocks_per_sm(c->nb, c->march_agg, c->march_minb, c->march_threads, 1);
    c->march_blocks = std::max(1, dev_sms * std::max(per_sm, 1));
    c->chem_blocks = std::max(1, (int)std::min<long long>((c->ncell + 255) / 256, (long long)dev_sms * 8));
    *out = c;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_add_sources(flexrt_ctx *c, int32_t n, const int32_t *ijk, const double *ndot) {
    if (!c) return FLEXRT_E_INVALID;
    if (n < 0 || (n > 0 && (!ijk || !ndot))) return c->fail(FLEXRT_E_INVALID, "bad source arrays");
    for (int32_t s = 0; s < n; ++s) {
        const int32_t *q = ijk + 3 * s;
        if (q[0] < 0 || q[0] >= c->h.nx || q[1] < 0 || q[1] >= c->h.ny || q[2] < 0 || q[2] >= c->h.nz ||
            !(ndot[s] >= 0.0))
            return c->fail(FLEXRT_E_INVALID, "source outside the grid or negative rate");
    }
    CK(c, cudaStreamSynchronize(c->st));
    size_t old = c->hcell.size();
    for (int32_t s = 0; s < n; ++s) {
        const int32_t *q = ijk + 3 * s;
        size_t f = c->hcell.size();
        for (size_t k = 0; k < c->hcell.size(); ++k)
            if (c->hcell[k].x == q[0] && c->hcell[k].y == q[1] && c->hcell[k].z == q[2]) { f = k; break; }
        if (f < c->hcell.size()) c->hndot[f] += ndot[s];
        else { c->hcell.push_back(make_int4(q[0], q[1], q[2], 0)); c->hndot.push_back(ndot[s]); }
    }
    const int ne = (int)c->hcell.size();
    if (!c->nref_set && ne > 0) {
        double mx = *std::max_element(c->hndot.begin(), c->hndot.end());
        if (mx > 0) {
            double r = mx * MYR_S * c->h.inv_ncast;
            c->h.nref = std::ldexp(1.0, (int)std::lround(std::log2(r)));
            c->nref_set = true;
            CK(c, cudaMemcpyAsync((char *)c->sims + offsetof(SimDev, nref), &c->h.nref, sizeof(double),
                                  cudaMemcpyHostToDevice, c->st));
        }
    }
    if (ne > c->ecap) {
        int cap = std::max(ne, std::max(16, 2 * c->ecap));
        Emitters ne_{};
        ne_.ring_w = c->em.ring_w;
        if (cudaMalloc(&ne_.cell, cap * sizeof(int4)) != cudaSuccess ||
            cudaMalloc(&ne_.local, cap * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&ne_.ndot, cap * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&ne_.n0, cap * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&ne_.ring, (size_t)cap * ne_.ring_w * 3 * sizeof(int4)) != cudaSuccess ||
            cudaMalloc(&ne_.act, cap * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&ne_.act_off, cap * sizeof(long long)) != cudaSuccess) {
            cudaFree(ne_.cell); cudaFree(ne_.local); cudaFree(ne_.ndot); cudaFree(ne_.n0);
            cudaFree(ne_.ring); cudaFree(ne_.act); cudaFree(ne_.act_off);
            return c->fail(FLEXRT_E_OOM, "emitter table allocation failed");
        }
        if (c->ecap > 0) {
            CK(c, cudaMemcpyAsync(ne_.ring, c->em.ring, (size_t)c->ecap * ne_.ring_w * 3 * sizeof(int4),
                                  cudaMemcpyDeviceToDevice, c->st));
            CK(c, cudaMemcpyAsync(ne_.n0, c->em.n0, c->ecap * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
            CK(c, cudaStreamSynchronize(c->st));
        }
        cudaFree(c->em.cell); cudaFree(c->em.local); cudaFree(c->em.ndot); cudaFree(c->em.n0);
        cudaFree(c->em.ring); cudaFree(c->em.act); cudaFree(c->em.act_off);
        c->em = ne_;
        c->ecap = cap;
    }
    (void)old;
    std::vector<int32_t> local(ne), act(ne);
    std::vector<long long> off(ne);
    const long long ncast = 12LL << (2 * c->h.l_src);
    for (int k = 0; k < ne; ++k) { local[k] = k; act[k] = k; off[k] = ncast * k; }
    CK(c, cudaMemcpyAsync(c->em.cell, c->hcell.data(), ne * sizeof(int4), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->em.ndot, c->hndot.data(), ne * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->em.local, local.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->em.act, act.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->em.act_off, off.data(), ne * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    long long et = ncast * ne;
    int32_t na = ne;
    CK(c, cudaMemcpyAsync((char *)c->ctl + offsetof(Ctl, emit_total), &et, sizeof(et), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync((char *)c->ctl + offsetof(Ctl, n_act_emit), &na, sizeof(na), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return FLEXRT_OK;
}

static flexrt_status poll_error(flexrt_ctx *c, bool wait) {
    if (c->latched != FLEXRT_OK) return c->latched;
    if (!c->err_pending) return FLEXRT_OK;
    if (wait) {
        cudaError_t e = cudaEventSynchronize(c->ev_err);
        if (e != cudaSuccess) return c->cuda(e, "step");
    } else if (cudaEventQuery(c->ev_err) != cudaSuccess) {
        return FLEXRT_OK;
    }
    c->err_pending = false;
    int32_t v = *c->h_err;
    if (v) {
        c->latched = FLEXRT_E_CAPACITY;
        if (v & 1) c->err = "ray queue capacity exceeded; state kept at the last complete step";
        else if (v & 2) c->err = "ray older than the rotation ring (internal bound)";
        else c->err = "ray crossed more than four cells in one step (internal bound)";
    }
    return c->latched;
}

static cudaEvent_t pool_event(flexrt_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

extern "C" flexrt_status flexrt_step(flexrt_ctx *c, double dt) {
    if (!c) return FLEXRT_E_INVALID;
    if (!(dt > 0.0)) return c->fail(FLEXRT_E_INVALID, "dt must be positive");
    flexrt_status s = poll_error(c, false);
    if (s != FLEXRT_OK) return s;
    if (dt != c->h.dt) {
        // wait until the previous dt upload has been consumed before reusing the slot
        CK(c, cudaEventSynchronize(c->ev_dt));
        c->h.dt = dt;
        c->h.gscale = c->h.nref * c->h.sigma_ref / (c->h.dx_phys * c->h.dx_phys * dt);
        c->h.hscale = c->h.gscale * EV_ERG;
        c->h_dt[0] = c->h.dt;
        c->h_dt[1] = c->h.gscale;
        c->h_dt[2] = c->h.hscale;
        static_assert(offsetof(SimDev, gscale) == offsetof(SimDev, dt) + sizeof(double), "dt/gscale layout");
        static_assert(offsetof(SimDev, hscale) == offsetof(SimDev, dt) + 2 * sizeof(double), "dt/hscale layout");
        CK(c, cudaMemcpyAsync((char *)c->sims + offsetof(SimDev, dt), c->h_dt, 3 * sizeof(double),
                              cudaMemcpyHostToDevice, c->st));
        CK(c, cudaEventRecord(c->ev_dt, c->st));
    }
    EmitArgs ea{c->ctl, c->sims, c->acc, {c->q[0], c->q[1]}, c->cap, c->em, c->pixtab, c->ltab, c->nb};
    MarchArgs ma{c->ctl, c->sims, c->acc, 1, {c->q[0], c->q[1]}, c->cap, c->em, c->cells, c->pixtab, c->ltab};
    ChemArgs ca{c->ctl, c->sims, c->acc, 1, c->cells, c->rg};
    const int ne = (int)c->hcell.size();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto tic = [&](int) {
        if (c->profiling) { e0 = pool_event(c); cudaEventRecord(e0, c->st); }
    };
    auto toc = [&](int k) {
        if (c->profiling) { e1 = pool_event(c); cudaEventRecord(e1, c->st); c->ev_k[k].push_back({e0, e1}); }
    };
    if (ne > 0) {
        tic(0);
        CK(c, launch_emit(ea, std::max(1, std::min((ne + 127) / 128, 1024)), c->st));
        toc(0);
    }
    tic(1);
    CK(c, launch_march(ma, c->nb, c->march_agg, c->march_minb, c->march_blocks, c->march_threads, c->st));
    toc(1);
    tic(2);
    CK(c, launch_chem(ca, c->chem_blocks, c->st));
    toc(2);
    CK(c, launch_end(c->ctl, c->sims, c->acc, 1, c->st));
    CK(c, cudaMemcpyAsync(c->h_err, (char *)c->ctl + offsetof(Ctl, err), sizeof(int32_t), cudaMemcpyDeviceToHost,
                          c->st));
    CK(c, cudaEventRecord(c->ev_err, c->st));
    c->err_pending = true;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_sync(flexrt_ctx *c) {
    if (!c) return FLEXRT_E_INVALID;
    CK(c, cudaStreamSynchronize(c->st));
    return poll_error(c, true);
}

extern "C" flexrt_status flexrt_reset(flexrt_ctx *c) {
    if (!c) return FLEXRT_E_INVALID;
    CK(c, cudaStreamSynchronize(c->st));
    c->latched = FLEXRT_OK;
    c->err_pending = false;
    int32_t zero = 0;
    long long z2[2] = {0, 0};
    CK(c, cudaMemcpyAsync((char *)c->ctl + offsetof(Ctl, cnt), z2, sizeof(z2), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync((char *)c->ctl + offsetof(Ctl, par), &zero, sizeof(zero), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync((char *)c->ctl + offsetof(Ctl, err), &zero, sizeof(zero), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync((char *)c->sims + offsetof(SimDev, step), &zero, sizeof(zero), cudaMemcpyHostToDevice, c->st));
    // keep the monotonic marched-ray counter (last field) for profiling windows
    CK(c, cudaMemsetAsync(c->acc, 0, offsetof(SimAcc, rays_in_total), c->st));
    CK(c, launch_init_cells(c->sims, 0, c->cells, c->ncell, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_get_fields(flexrt_ctx *c, flexrt_fields *f) {
    if (!c || !f) return FLEXRT_E_INVALID;
    CK(c, cudaStreamSynchronize(c->st));
    flexrt_status s = poll_error(c, true);
    if (s != FLEXRT_OK && s != FLEXRT_E_CAPACITY) return s;
    s = FLEXRT_OK;
    const size_t n = (size_t)c->ncell;
    std::vector<double> y;
    std::vector<float> t;
    if (f->T || f->gamma_HI || f->x_HII) t.resize(n);
    if (f->n_HI) {
        y.resize(n);
        CK(c, cudaMemcpy(y.data(), c->cells.y, n * sizeof(double), cudaMemcpyDeviceToHost));
        CK(c, cudaMemcpy(f->n_HI, c->cells.nH, n * sizeof(double), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) f->n_HI[i] *= y[i];
    }
    if (f->x_HII) {
        CK(c, cudaMemcpy(t.data(), c->cells.x, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) f->x_HII[i] = t[i];
    }
    if (f->T) {
        CK(c, cudaMemcpy(t.data(), c->cells.T, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) f->T[i] = t[i];
    }
    if (f->gamma_HI) {
        CK(c, cudaMemcpy(t.data(), c->cells.gamma, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) f->gamma_HI[i] = t[i];
    }
    return s;
}

static flexrt_status read_acc(flexrt_ctx *c, SimAcc &a) {
    CK(c, cudaStreamSynchronize(c->st));
    CK(c, cudaMemcpy(&a, c->acc, sizeof(a), cudaMemcpyDeviceToHost));
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_get_budget(flexrt_ctx *c, double out[4]) {
    if (!c || !out) return FLEXRT_E_INVALID;
    SimAcc a;
    flexrt_status s = read_acc(c, a);
    if (s != FLEXRT_OK) return s;
    const double r = c->h.nref;
    out[0] = a.emitted * r; out[1] = a.absorbed * r; out[2] = a.escaped * r; out[3] = a.in_flight * r;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_get_counts(flexrt_ctx *c, int64_t out[6]) {
    if (!c || !out) return FLEXRT_E_INVALID;
    SimAcc a;
    flexrt_status s = read_acc(c, a);
    if (s != FLEXRT_OK) return s;
    int32_t step = 0;
    CK(c, cudaMemcpy(&step, (char *)c->sims + offsetof(SimDev, step), sizeof(step), cudaMemcpyDeviceToHost));
    out[0] = (int64_t)a.rays_live; out[1] = (int64_t)a.seg_last; out[2] = (int64_t)a.seg_total;
    out[3] = step; out[4] = c->cap; out[5] = (int64_t)a.rays_in_last;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_get_segment_counts(flexrt_ctx *c, int32_t *out) {
    if (!c || !out) return FLEXRT_E_INVALID;
    if (!c->cells.segcnt) return c->fail(FLEXRT_E_STATE, "created without keep_diagnostics");
    CK(c, cudaStreamSynchronize(c->st));
    CK(c, cudaMemcpy(out, c->cells.segcnt, (size_t)c->ncell * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_get_rays(flexrt_ctx *c, int64_t cap, int32_t *level, int64_t *pixel,
                                         int32_t *emitter, int32_t *birth, int32_t *dir, double *photons,
                                         int64_t *n) {
    if (!c || !n || cap < 0) return FLEXRT_E_INVALID;
    CK(c, cudaStreamSynchronize(c->st));
    Ctl hc;
    CK(c, cudaMemcpy(&hc, c->ctl, sizeof(hc), cudaMemcpyDeviceToHost));
    SimAcc a;
    CK(c, cudaMemcpy(&a, c->acc, sizeof(a), cudaMemcpyDeviceToHost));
    *n = (int64_t)a.rays_live;
    const long long m = hc.cnt[hc.par];  // queue slots, live or unused
    if (m == 0 || cap == 0) return FLEXRT_OK;
    const Queue &q = c->q[hc.par];
    std::vector<uint32_t> pl(m), em(m);
    std::vector<int32_t> bi(m), d(3 * m);
    CK(c, cudaMemcpy(pl.data(), q.pl, m * 4, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(em.data(), q.em, m * 4, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(bi.data(), q.bi, m * 4, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(d.data(), q.dx, m * 4, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(d.data() + m, q.dy, m * 4, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(d.data() + 2 * m, q.dz, m * 4, cudaMemcpyDeviceToHost));
    std::vector<std::vector<float>> ph(photons ? c->nb : 0, std::vector<float>(m));
    for (int b = 0; b < (int)ph.size(); ++b)
        CK(c, cudaMemcpy(ph[b].data(), q.ph[b], m * 4, cudaMemcpyDeviceToHost));
    long long k = 0;  // live rays only: queue slots marked unused are skipped
    for (long long i = 0; i < m && k < cap; ++i) {
        if (pl[i] == DEAD_RAY) continue;
        if (level) level[k] = (int32_t)(pl[i] >> LEVEL_SHIFT);
        if (pixel) pixel[k] = (int64_t)(pl[i] & PIX_MASK);
        if (emitter) emitter[k] = (int32_t)em[i];
        if (birth) birth[k] = bi[i];
        if (dir) { dir[3 * k] = d[i]; dir[3 * k + 1] = d[m + i]; dir[3 * k + 2] = d[2 * m + i]; }
        for (int b = 0; b < (int)ph.size(); ++b) photons[(size_t)c->nb * k + b] = (double)ph[b][i] * c->h.nref;
        ++k;
    }
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_profile(flexrt_ctx *c, int32_t enable) {
    if (!c) return FLEXRT_E_INVALID;
    double dummy[3];
    int64_t l[3], r[1];
    flexrt_status s = flexrt_get_kernel_times(c, dummy, l, r);
    c->profiling = enable != 0;
    return s;
}

extern "C" flexrt_status flexrt_get_kernel_times(flexrt_ctx *c, double ms[3], int64_t launches[3],
                                                 int64_t march_rays[1]) {
    if (!c || !ms || !launches) return FLEXRT_E_INVALID;
    CK(c, cudaStreamSynchronize(c->st));
    for (int k = 0; k < 3; ++k) {
        double t = 0.0;
        for (auto &p : c->ev_k[k]) {
            float x = 0.f;
            cudaEventElapsedTime(&x, p.first, p.second);
            t += x;
            c->ev_pool.push_back(p.first);
            c->ev_pool.push_back(p.second);
        }
        ms[k] = t;
        launches[k] = (int64_t)c->ev_k[k].size();
        c->ev_k[k].clear();
    }
    SimAcc a;
    flexrt_status s = read_acc(c, a);
    if (s != FLEXRT_OK) return s;
    if (march_rays) march_rays[0] = (int64_t)(a.rays_in_total - c->rays_total_at_profile);
    c->rays_total_at_profile = a.rays_in_total;
    return FLEXRT_OK;
}

extern "C" flexrt_status flexrt_set_launch(flexrt_ctx *c, int32_t agg, int32_t minb, int32_t blocks_per_sm) {
    if (!c) return FLEXRT_E_INVALID;
    if (!march_variant_exists(c->nb, agg, minb) || blocks_per_sm < 0 || blocks_per_sm > 32)
        return c->fail(FLEXRT_E_INVALID, "march kernel variant not built");
    int lim = march_max_blocks_per_sm(c->nb, agg, minb, c->march_threads, 1);
    if (lim < 1) return c->fail(FLEXRT_E_INVALID, "variant cannot be resident");
    int bps = blocks_per_sm == 0 ? lim : std::min(blocks_per_sm, lim);
    c->march_agg = agg;
    c->march_minb = minb;
    c->march_blocks = c->sm_count * bps;
    return FLEXRT_OK;
}

namespace frt {
static thread_local std::string g_free_err;
void set_free_error(const std::string &msg) { g_free_err = msg; }
}  // namespace frt

extern "C" const char *flexrt_last_error(const flexrt_ctx *c) {
    return c ? c->err.c_str() : frt::g_free_err.c_str();
}

extern "C" void flexrt_destroy(flexrt_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    free_ctx(c);
}

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
