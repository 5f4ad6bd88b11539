// frt_march.cuh -- the fused per-ray kernel of one RT step, shared by the
// translation unit that builds the plain variants and the one that builds
// the variants carrying merged rays.
//
//   k_march : per ray, the one-cell march with exp(-tau) attenuation
//             (Sec. 3.1; Sec. 4.2, Eq. 13), the Eq. 17 deposit (warp-aggregated
//             vector reductions into the per-cell buffers), escape,
//             termination, the Eq. 2-3 split and the compacted write of
//             survivors and children.
#pragma once
#include "frt_device.cuh"
#include "frt_launch.h"

namespace frt {

constexpr int NACC = 6;  // (unused), escaped, out, segments, rays in, rays out

// Warp-wide flush of lane-private tallies (lane simulation `tsim`, -1 for
// none) into the block's per-simulation fixed-point totals; clears them.
__device__ __forceinline__ void flush_tallies(float &esc, float &out, unsigned &cnt, unsigned &rout, int &tsim,
                                              unsigned long long *sh_acc) {
    const int lane = lane_id();
    const int kref = __reduce_max_sync(FULL, tsim);
    if (kref < 0) return;                                   // warp-uniform
    float v[NACC] = {0.0f, esc, out, (float)(cnt & 0xffffu), (float)(cnt >> 16), (float)rout};
    bool lead;
    int kk = tsim;
    if (__all_sync(FULL, tsim < 0 || tsim == kref)) {
        warp_sum<NACC>(v);                                  // empty lanes carry zeros
        lead = lane == 0;
        kk = kref;
    } else {
        const unsigned peers = __match_any_sync(FULL, tsim);
        peer_sum<NACC>(peers, v);
        lead = tsim >= 0 && (peers & ((1u << lane) - 1u)) == 0u;
    }
    if (lead) {
        unsigned long long *dst = sh_acc + kk * NACC;
        atomicAdd(dst + 0, fixed32(v[0]));
        atomicAdd(dst + 1, fixed32(v[1]));
        atomicAdd(dst + 2, fixed32(v[2]));
        atomicAdd(dst + 3, (unsigned long long)__float2uint_rn(v[3]));
        atomicAdd(dst + 4, (unsigned long long)__float2uint_rn(v[4]));
        atomicAdd(dst + 5, (unsigned long long)__float2uint_rn(v[5]));
    }
    esc = out = 0.0f;
    cnt = rout = 0u;
    tsim = -1;
}

// The per-simulation constants the march needs, staged in shared memory.
struct MarchSim {
    int nx, ny, nz, step, l_src, l_max, active, l_merge, gen, pad0, pad1, pad2;
    long long coff;
    float eps;
    float sig_max;          // largest sigma_b / sigma_ref of the bins
    int K[MAXL];
    float sig[MAXB], sige[MAXB], eh[MAXB];
};

__host__ __device__ constexpr size_t march_shared_bytes(int nsims) {
    return (size_t)nsims * (NACC * sizeof(unsigned long long) + sizeof(MarchSim));
}

// (1 - e^-t)/t for 0 <= t < 1/8: its Taylor series through t^4 (the next
// term, t^5/720, is under the single-precision epsilon there)
__device__ __forceinline__ float2 series_q2(float2 t) {
    const float2 nt = make_float2(-t.x, -t.y);
    float2 q = make_float2(1.0f / 120.0f, 1.0f / 120.0f);
    q = __ffma2_rn(q, nt, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
    q = __ffma2_rn(q, nt, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
    q = __ffma2_rn(q, nt, make_float2(0.5f, 0.5f));
    return __ffma2_rn(q, nt, make_float2(1.0f, 1.0f));
}
__device__ __forceinline__ float series_q(float t) {
    float q = 1.0f / 120.0f;
    q = fmaf(q, -t, 1.0f / 24.0f);
    q = fmaf(q, -t, 1.0f / 6.0f);
    q = fmaf(q, -t, 0.5f);
    return fmaf(q, -t, 1.0f);
}

// Attenuation of the photons ph[b] entering a segment of length dse (cells)
// through a cell of optical depth per cell k = (HI at sigma_ref, sub-grid),
// with its deposits (Eq. 13, Eq. 17): v[0] += absorbed photons, v[1] +=
// sum_b sigma_b N_b (1 - e^-tau_b)/kappa_b, v[2] the same weighted by the
// excess energy.  A bin with tau < 1/8 takes 1 - e^-tau = tau q(tau) with
// the series q, so (1 - e^-tau)/kappa = dse q (no exponential, no
// division) and keeps N - N tau q; a thicker bin takes the hardware
// exponential and the division by kappa (N dse when kappa = 0).  SMALL:
// every bin of every lane of the warp is thin, and only the series is
// evaluated; the per-bin results are the same either way, so a ray's photons
// do not depend on the rays it shares a warp with.  Bins go in pairs on the
// paired single-precision units.
template <int NB, bool SMALL>
__device__ __forceinline__ void seg_attenuate(float2 k, float dse, const float *sig, const float *sige, float (&ph)[NB],
                                              float (&v)[4]) {
    float2 w0 = make_float2(0.f, 0.f), w1 = w0, w2 = w0;
    const float2 kx2 = make_float2(k.x, k.x), ky2 = make_float2(k.y, k.y), ds2 = make_float2(dse, dse);
#pragma unroll
    for (int b = 0; b + 1 < NB; b += 2) {
        const float2 sg = make_float2(sig[b], sig[b + 1]);
        const float2 se = make_float2(sige[b], sige[b + 1]);
        const float2 kb = __ffma2_rn(kx2, sg, ky2);
        const float2 tau = __fmul2_rn(kb, ds2);
        const float2 p2 = make_float2(ph[b], ph[b + 1]);
        const float2 pd = __fmul2_rn(p2, ds2);
        float2 a, phin, pn;
        if (SMALL) {
            const float2 q = series_q2(tau);
            a = __fmul2_rn(p2, __fmul2_rn(q, tau));
            phin = __fmul2_rn(pd, q);
            pn = __fadd2_rn(p2, make_float2(-a.x, -a.y));
        } else {
            const float2 u = make_float2(fminf(tau.x, 0.125f), fminf(tau.y, 0.125f));
            const float2 q = series_q2(u);
            const float2 as = __fmul2_rn(p2, __fmul2_rn(q, u));
            const float2 ps = __fmul2_rn(pd, q);
            const float ex0 = __expf(-tau.x), ex1 = __expf(-tau.y);
            const bool s0 = tau.x < 0.125f, s1 = tau.y < 0.125f;
            a = make_float2(s0 ? as.x : p2.x * (1.0f - ex0), s1 ? as.y : p2.y * (1.0f - ex1));
            pn = make_float2(s0 ? p2.x - as.x : p2.x * ex0, s1 ? p2.y - as.y : p2.y * ex1);
            phin = make_float2(s0 ? ps.x : (kb.x > 0.0f ? __fdividef(a.x, kb.x) : pd.x),
                               s1 ? ps.y : (kb.y > 0.0f ? __fdividef(a.y, kb.y) : pd.y));
        }
        ph[b] = pn.x;
        ph[b + 1] = pn.y;
        w0 = __fadd2_rn(w0, a);
        w1 = __ffma2_rn(sg, phin, w1);
        w2 = __ffma2_rn(se, phin, w2);
    }
    v[0] = w0.x + w0.y;
    v[1] = w1.x + w1.y;
    v[2] = w2.x + w2.y;
    if (NB & 1) {
        const int b = NB - 1;
        const float kb = fmaf(k.x, sig[b], k.y);
        const float tau = kb * dse;
        const float pd = ph[b] * dse;
        float a, phin;
        if (SMALL || tau < 0.125f) {
            const float q = series_q(tau);
            a = ph[b] * (q * tau);
            phin = pd * q;
            ph[b] -= a;
        } else {
            const float ex = __expf(-tau);
            a = ph[b] * (1.0f - ex);
            phin = kb > 0.0f ? __fdividef(a, kb) : pd;
            ph[b] *= ex;
        }
        v[0] += a;
        v[1] = fmaf(sig[b], phin, v[1]);
        v[2] = fmaf(sige[b], phin, v[2]);
    }
}

// Phases per ray: (1) the integer walk of the whole step, (2) the opacity
// loads of every crossed cell at once, (3) attenuation and deposits.
// AGG selects how the lanes of a warp combine deposits into the same cell
// before the vector reduction: 0 none, 1 peer groups of equal keys
// (match_any + pairwise tree), 2 runs of equal consecutive keys.
// MINB is the resident-block target per SM (register budget).  EXT bit 1
// adds the rays made by the merge step (Sec. 3.3), which start from their
// merge position and carry their own distance and termination threshold;
// bit 2 adds Generalized Opacity mode (Sec. 4.2): a ray crosses the ionised
// fraction x_ion of each cell's path with the sub-grid opacity, then meets
// the moving screen, which absorbs the share rho of what reaches it
// (Eq. 18-19).  A merging engine without Generalized members runs EXT = 1
// (fewer registers: 10% less march time on the merging workloads than with
// both), an engine that may run Generalized members EXT = 3.
template <int NB, int AGG, int MINB, int EXT>
__global__ void __launch_bounds__(256, MINB) k_march(MarchArgs A) {
    constexpr bool MRG = (EXT & 1) != 0, GEN = (EXT & 2) != 0;
    // per-simulation tallies of this block (photons in 2^-32 fixed point,
    // counts as integers), then the staged constants
    extern __shared__ unsigned long long sh_acc[];
    MarchSim *msim = reinterpret_cast<MarchSim *>(sh_acc + A.nsims * NACC);
    for (int i = threadIdx.x; i < A.nsims * NACC; i += blockDim.x) sh_acc[i] = 0ull;
    for (int i = threadIdx.x; i < A.nsims; i += blockDim.x) {
        const SimDev &S = A.sims[i];
        MarchSim &m = msim[i];
        m.nx = S.nx; m.ny = S.ny; m.nz = S.nz; m.step = S.step; m.l_src = S.l_src; m.l_max = S.l_max;
        m.active = S.active; m.l_merge = S.l_merge; m.coff = S.cell_off; m.eps = S.eps_term;
        m.gen = S.gen_mode; m.pad0 = m.pad1 = m.pad2 = 0;
        for (int l = 0; l < MAXL; ++l) m.K[l] = S.K[l];
        m.sig_max = 0.0f;
        for (int b = 0; b < MAXB; ++b) {
            m.sig[b] = S.sig[b]; m.sige[b] = S.sige[b]; m.eh[b] = S.eh[b];
            if (b < S.nb) m.sig_max = fmaxf(m.sig_max, S.sig[b]);
        }
    }
    __syncthreads();
    Ctl *C = A.ctl;
    const int lane = lane_id();
    if (C->err == 0) {
        const int par = C->par;
        const Queue qi = A.q[par], qo = A.q[par ^ 1];
        unsigned long long *out_cnt = (unsigned long long *)&C->cnt[par ^ 1];
        // queue slots stay below 2^31 (the engine's bound), so 32-bit indices
        const unsigned n = (unsigned)(C->cnt[par] + C->emit_total);
        const unsigned nr = (n + 31u) & ~31u;
        const unsigned stride = gridDim.x * blockDim.x;
        // warp-private run of output slots [slab, slab + slab_left), and this
        // warp's outputs and iterations so far (its output rate)
        unsigned slab = 0;
        int slab_left = 0;
        int w_out = 0, w_it = 0;
        // lane-private tallies of one simulation, flushed by the warp:
        // escaped and surviving photons, segments | rays in << 16, rays out
        float t_esc = 0.0f, t_out = 0.0f;
        unsigned t_cnt = 0u, t_rout = 0u;
        int t_sim = -1, t_n = 0;
        // the ray's words, loaded at the top of its iteration (loading the next
        // ray's one iteration ahead cost more in spilled registers than it hid)
        uint32_t npl = DEAD_RAY, ne_ = 0;
        int nbi = 0, ndx = 0, ndy = 0, ndz = 0;
        float nph[NB];
        int nmx = 0, nmy = 0, nmz = 0;
        uint32_t nma = 0;
        float nmthr = 0.0f;
        auto load_ray = [&](unsigned j) {
            // the queue streams through once per step: evict-first loads keep
            // the cells' opacities and deposit buffers resident in L2
            npl = DEAD_RAY;
            if (j < n) npl = __ldcs(qi.pl + j);
            if (npl != DEAD_RAY) {
                ne_ = __ldcs(qi.em + j); nbi = __ldcs(qi.bi + j);
                ndx = __ldcs(qi.dx + j); ndy = __ldcs(qi.dy + j); ndz = __ldcs(qi.dz + j);
#pragma unroll
                for (int b = 0; b < NB; ++b) nph[b] = __ldcs(qi.ph[b] + j);
                if (MRG && (ne_ & MERGED_BIT)) {
                    nmx = __ldcs(qi.mx + j); nmy = __ldcs(qi.my + j); nmz = __ldcs(qi.mz + j);
                    nma = __ldcs(qi.ma + j); nmthr = __ldcs(qi.mthr + j);
                }
            } else {
                ne_ = 0; nbi = 0; ndx = ndy = ndz = 0;
#pragma unroll
                for (int b = 0; b < NB; ++b) nph[b] = 0.0f;
            }
        };
        for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
            load_ray(i);
            const uint32_t pl = npl, e = ne_;
            const int bi = nbi, dx = ndx, dy = ndy, dz = ndz;
            const int mx = nmx, my = nmy, mz = nmz;
            const uint32_t ma = nma;
            const float mthr = nmthr;
            float ph[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) ph[b] = nph[b];
            bool valid = pl != DEAD_RAY;
            const bool mrg = MRG && valid && (e & MERGED_BIT);
            int sim = 0;
            int4 ec = make_int4(0, 0, 0, 0);
            if (mrg) {
                sim = (int)((ma >> 16) & 0x7fffu);
            } else if (valid) {
                ec = __ldg(&A.em.cell[e]);
                sim = ec.w;
            }
            const MarchSim &S = msim[sim];
            if (!S.active) valid = false;
            // age: cells travelled before this step.  A merged ray has moved
            // `since` steps from its merge position and had travelled its
            // constituents' mean distance when it was made.
            const int since = S.step - bi - 1;
            const int age = mrg ? (int)(ma & 0xffffu) + since : S.step - bi;
            if (valid && (mrg ? since < 0 : (age < 0 || age >= A.em.ring_w))) {
                atomicOr(&C->err, 2);
                valid = false;
            }

            // (1) integer walk of this step
            int key[4];
            float ds[4];
            bool esc = false;
            int nseg = 0;
            unsigned vmask = 0u;
            {
                Walk w;
                // a queued ray is inside the box at the start of its step, so
                // its position (at most 1000 cells of 2^21) fits 32 bits
                int px, py, pz;
                if (mrg) {
                    px = mx + since * dx;
                    py = my + since * dy;
                    pz = mz + since * dz;
                } else {
                    px = ((2 * ec.x + 1) << (FRAC_BITS - 1)) + age * dx;
                    py = ((2 * ec.y + 1) << (FRAC_BITS - 1)) + age * dy;
                    pz = ((2 * ec.z + 1) << (FRAC_BITS - 1)) + age * dz;
                }
                walk_init(w, px, py, pz, dx, dy, dz);
                // slots may be empty (tied crossings): every later phase
                // visits the four slots in order and skips the empty ones
#pragma unroll
                for (int j = 0; j < 4; ++j) { key[j] = -1; ds[j] = 0.0f; }
                if (valid) vmask = walk_step(w, S.nx, S.ny, S.nz, (int)S.coff, key, ds, esc);
                nseg = __popc(vmask);
            }
            // (2) opacities of the crossed cells (Generalized mode: also the
            // ionised fraction and the screen's share)
            float2 kc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) kc[j] = key[j] >= 0 ? __ldg(&A.cells.kap[key[j]]) : make_float2(0.f, 0.f);
            const bool gen = GEN && valid && S.gen;
            float xg[4], rg[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xg[j] = 1.0f;
                rg[j] = 1.0f;
                if (GEN && gen && key[j] >= 0) { xg[j] = (float)__ldg(&A.cells.xion[key[j]]); rg[j] = __ldg(&A.cells.rho[key[j]]); }
            }
            bool screened = false;
            // (3) attenuation and deposits (Eq. 13, Eq. 17)
            int last = -1;
            float2 lastk = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float v[4] = {0.f, 0.f, 0.f, 1.0f};
                if (GEN && screened) key[j] = -1;
                const float dse = GEN ? xg[j] * ds[j] : ds[j];
                // every segment of this slot in the warp optically thin (all
                // bins' tau below 1/8): the series path, warp-uniform
                const bool thin = __all_sync(FULL, key[j] < 0 || fmaf(kc[j].x, S.sig_max, kc[j].y) * dse < 0.125f);
                if (key[j] >= 0) {
                    if (thin) seg_attenuate<NB, true>(kc[j], dse, S.sig, S.sige, ph, v);
                    else seg_attenuate<NB, false>(kc[j], dse, S.sig, S.sige, ph, v);
                    last = key[j];
                    lastk = kc[j];
                    if (GEN && xg[j] < 1.0f) {
                        // the screen: it absorbs the share rho of what reaches it
                        float nf = 0.0f;
#pragma unroll
                        for (int b = 0; b < NB; ++b) nf += ph[b];
                        red_add_v2(A.cells.fscr + key[j], rg[j] * nf, nf);
                        const float keep = rg[j] >= 1.0f ? 0.0f : 1.0f - rg[j];
#pragma unroll
                        for (int b = 0; b < NB; ++b) ph[b] *= keep;
                        if (rg[j] >= 1.0f) {
                            screened = true;
                            nseg = __popc(vmask & ((2u << j) - 1u));
                        }
                    }
                }
                if (AGG == 0) {
                    if (key[j] >= 0) red_add_v4(A.cells.dep + key[j], v[0], v[1], v[2], v[3]);
                } else {
                    if (__ballot_sync(FULL, key[j] >= 0) == 0u) continue;
                    if (AGG == 1) {
                        const unsigned peers = __match_any_sync(FULL, key[j]);
                        if (__any_sync(FULL, key[j] >= 0 && __popc(peers) > 1)) peer_sum<4>(peers, v);
                        if (key[j] >= 0 && (peers & ((1u << lane) - 1u)) == 0u)
                            red_add_v4(A.cells.dep + key[j], v[0], v[1], v[2], v[3]);
                    } else {
                        const bool head = run_sum<4>(key[j], v);
                        if (key[j] >= 0 && head) red_add_v4(A.cells.dep + key[j], v[0], v[1], v[2], v[3]);
                    }
                }
            }
            float s_end = 0.0f;
#pragma unroll
            for (int b = 0; b < NB; ++b) s_end += ph[b];
            int nout = 0, m = 0;
            const int lev = (int)(pl >> LEVEL_SHIFT);
            if (GEN && screened) esc = false;
            if (valid && !esc && !(GEN && screened)) {
                const float thr = mrg ? mthr : S.eps * __ldg(&A.em.n0[e]) * pow2_neg(2 * (lev - S.l_src));
                if (s_end < thr) {
                    // termination: the ray's last photons stay in its last cell
                    float g = 0.f, h = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const float kb = fmaf(lastk.x, S.sig[b], lastk.y);
                        if (kb > 0.0f) {
                            const float q = __fdividef(ph[b], kb);
                            g = fmaf(S.sig[b], q, g);
                            h = fmaf(S.sige[b], q, h);
                        }
                    }
                    red_add_v4(A.cells.dep + last, s_end, g, h, 0.0f);
                } else {
                    while (lev + m < S.l_max && age + 1 >= S.K[lev + m]) ++m;
                    nout = 1 << (2 * m);
                }
            }
            // per-simulation tallies: each lane accumulates the rays of one
            // simulation for up to sixteen iterations, then the warp reduces them
            // into the block's fixed-point totals
            {
                const bool clash = valid && t_sim >= 0 && t_sim != sim;
                if (__any_sync(FULL, clash) || t_n == 16) {
                    flush_tallies(t_esc, t_out, t_cnt, t_rout, t_sim, sh_acc);
                    t_n = 0;
                }
                if (valid) {
                    if (esc) t_esc += s_end;
                    if (nout) t_out += s_end;
                    t_cnt += (unsigned)nseg + (1u << 16);
                    t_rout += (unsigned)nout;
                    t_sim = sim;
                }
                ++t_n;
            }
            // compacted output into the warp's run of slots: the remainder of
            // the current run first, then a new run reserved with one atomic
            const int incl = warp_incl_scan(nout);
            const int tot = __shfl_sync(FULL, incl, 31);
            if (tot > 0) {
                const unsigned s0 = slab;
                const int left = slab_left;
                unsigned s1 = 0;
                bool fits = true;
                if (tot > left) {
                    // reserve for this warp's next iterations at its own output
                    // rate (at most 16 iterations ahead and OUT_SLAB slots), so the
                    // unused tail stays small whatever the queue's dead fraction
                    const int need = tot - left;
                    const unsigned iters_left = (nr - i + stride - 1u) / stride;
                    const int ahead = iters_left < 16u ? (int)iters_left : 16;
                    const int rate = (w_out + tot + w_it) / (w_it + 1);
                    const int guess = rate * ahead < A.slab ? rate * ahead : A.slab;
                    const int want = need > guess ? need : guess;
                    unsigned long long nb64 = 0;
                    if (lane == 0) nb64 = atomicAdd(out_cnt, (unsigned long long)want);
                    nb64 = __shfl_sync(FULL, nb64, 0);
                    const unsigned nbase = (unsigned)nb64;
                    if ((long long)(nb64 + want) > A.cap) {
                        if (lane == 0) atomicOr(&C->err, 1);
                        fits = false;
                        slab_left = 0;
                    } else {
                        s1 = nbase;
                        slab = nbase + need;
                        slab_left = want - need;
                    }
                } else {
                    slab = s0 + tot;
                    slab_left = left - tot;
                }
                w_out += tot;
                if (fits && nout > 0) {
                    const int k0 = incl - nout;  // this lane's first output position
                    auto slot_of = [&](int k) -> unsigned {
                        return k < left ? s0 + (unsigned)k : s1 + (unsigned)(k - left);
                    };
                    if (nout == 1) {
                        const unsigned o = slot_of(k0);
                        __stcs(qo.pl + o, pl); __stcs(qo.em + o, e); __stcs(qo.bi + o, bi);
                        __stcs(qo.dx + o, dx); __stcs(qo.dy + o, dy); __stcs(qo.dz + o, dz);
#pragma unroll
                        for (int b = 0; b < NB; ++b) __stcs(qo.ph[b] + o, ph[b]);
                        if (mrg) {
                            __stcs(qo.mx + o, mx); __stcs(qo.my + o, my); __stcs(qo.mz + o, mz);
                            __stcs(qo.ma + o, ma); __stcs(qo.mthr + o, mthr);
                        }
                    } else {
                        const int L = lev + m;
                        const uint32_t pix0 = (pl & PIX_MASK) << (2 * m);
                        // children keep their parent's sphere (Sec. 3.2): the
                        // emitter's of the birth step, or the merge cell's
                        int4 rows[3];
                        if (mrg) {
                            const SimDev &SD = A.sims[sim];
                            rotation_rows(SD.seed, (1LL << 31) + (long long)(e & ~MERGED_BIT), bi, SD.rotate, rows);
                        } else {
                            const int4 *rg = A.em.ring + ((long long)e * A.em.ring_w + (bi % A.em.ring_w)) * 3;
                            rows[0] = rg[0]; rows[1] = rg[1]; rows[2] = rg[2];
                        }
                        const bool vert = mrg && (ma >> 31);
                        const float scale = pow2_neg(2 * m);
                        float cph[NB];
#pragma unroll
                        for (int b = 0; b < NB; ++b) cph[b] = ph[b] * scale;
                        for (int c = 0; c < nout; ++c) {
                            const uint32_t pix = vert ? vertex_child(S.l_merge, pl & PIX_MASK, lev, m, (uint32_t)c)
                                                      : pix0 + (uint32_t)c;
                            const int4 vq = L <= A.ltab ? __ldg(&A.pixtab[level_offset(L) + pix]) : healpix_vq(L, pix);
                            int32_t cx, cy, cz;
                            rotate_dir(rows, vq, cx, cy, cz);
                            const unsigned oc = slot_of(k0 + c);
                            qo.pl[oc] = ((uint32_t)L << LEVEL_SHIFT) | pix;
                            qo.em[oc] = e; qo.bi[oc] = bi;
                            qo.dx[oc] = cx; qo.dy[oc] = cy; qo.dz[oc] = cz;
#pragma unroll
                            for (int b = 0; b < NB; ++b) qo.ph[b][oc] = cph[b];
                            if (mrg) {
                                qo.mx[oc] = mx; qo.my[oc] = my; qo.mz[oc] = mz;
                                qo.ma[oc] = ma & 0x7fffffffu;
                                qo.mthr[oc] = mthr * scale;
                            }
                        }
                    }
                }
            }
            ++w_it;
        }
        for (int k = lane; k < slab_left; k += 32) qo.pl[slab + k] = DEAD_RAY;
        flush_tallies(t_esc, t_out, t_cnt, t_rout, t_sim, sh_acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < A.nsims * NACC; i += blockDim.x) {
        const unsigned long long u = sh_acc[i];
        const double v = (i % NACC) < 3 ? (double)u * 0x1p-32 : (double)u;
        if (u != 0ull) {
            SimAcc &a = A.acc[i / NACC];
            double *dst = nullptr;
            switch (i % NACC) {
                case 0: dst = &a.p_in; break;
                case 1: dst = &a.p_esc; break;
                case 2: dst = &a.p_out; break;
                case 3: dst = &a.p_seg; break;
                case 4: dst = &a.p_rays_in; break;
                default: dst = &a.p_rays_out; break;
            }
            atomicAdd(dst, v);
        }
    }
}

}  // namespace frt
