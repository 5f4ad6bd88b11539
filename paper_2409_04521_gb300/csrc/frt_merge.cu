// frt_merge.cu -- ray merging at the end of a step (Sec. 3.3, Eq. 4) and the
// march variants that carry merged rays.
//
// The step, per simulation that merges (it has more live rays than
// K = floor(N_ex * N_RT)):
//   k_mrot    : per cell, the random rotation of the cell's merge sphere for
//               this step, drawn like an emitter's sphere (key 2^31 + local
//               cell index; exact integer arithmetic);
//   k_mhist1  : per ray, its content (single-precision sum of its bins, the
//               quantity ranked) and a histogram of the content's upper 16 bits;
//   k_mfind   : per simulation, a two-pass radix select of the K-th largest
//               content T_ref (the largest when K = 0): with K > 0 every ray
//               at least that bright is exempt;
//   k_mhist2  : per ray in the selected upper bin, a histogram of the lower bits;
//   k_mgroup  : per non-exempt ray, its end cell and merge pixel; a group slot
//               per (cell, pixel) takes its photons and threshold (vector
//               reductions), the largest member content and the ray's arrival
//               rank: rank 0 leads the group and is listed, the others leave
//               the queue (their slots become holes); the ray's group slot and
//               its end point, distance and level are kept per queue slot;
//   k_mweight : per grouped ray, its photon weight -- the content on a grid of
//               2^-28 of the power of two above its group's largest content,
//               truncated, at least 1 -- and the weighted end point, distance
//               and level as exact 64-bit integer sums, so the photon-weighted
//               means are exact quotients of sums that do not depend on the
//               summation order, to 2^-27 of the group's brightest member;
//   k_memit   : per listed leader: it overwrites its own slot with the merged
//               ray (means rounded once) and clears the group.
// The holes stay in the queue: the next march skips them and writes its
// survivors densely into the other queue, so no compaction pass is needed.
// Contents are non-negative floats, so their bit patterns order as unsigned
// integers and the select and the group maximum work on the bits.
#include "frt_march.cuh"

namespace frt {

// ---------------------------------------------------------------------------
// march variants with merged rays
// ---------------------------------------------------------------------------
MarchFn march_fn_merge(int nb, int agg, int minb) {
#define FRT_V(NB)                                                                   \
    if (nb == NB) {                                                                \
        if (agg == 0 && minb == 2) return k_march<NB, 0, 2, 1>;                    \
        if (agg == 0 && minb == 3) return k_march<NB, 0, 3, 1>;                    \
        if (agg == 0 && minb == 4) return k_march<NB, 0, 4, 1>;                    \
        if (agg == 1 && minb == 2) return k_march<NB, 1, 2, 1>;                    \
        if (agg == 1 && minb == 3) return k_march<NB, 1, 3, 1>;                    \
        if (agg == 1 && minb == 4) return k_march<NB, 1, 4, 1>;                    \
        if (agg == 2 && minb == 2) return k_march<NB, 2, 2, 1>;                    \
        if (agg == 2 && minb == 3) return k_march<NB, 2, 3, 1>;                    \
        if (agg == 2 && minb == 4) return k_march<NB, 2, 4, 1>;                    \
        return nullptr;                                                            \
    }
    FRT_V(1)
    FRT_V(3)
    FRT_V(4)
#undef FRT_V
    if (agg != 0 || minb != 2) return nullptr;
    switch (nb) {
        case 2: return k_march<2, 0, 2, 1>;
        case 5: return k_march<5, 0, 2, 1>;
        case 6: return k_march<6, 0, 2, 1>;
        case 7: return k_march<7, 0, 2, 1>;
        case 8: return k_march<8, 0, 2, 1>;
        default: return nullptr;
    }
}

namespace {

// per-simulation selection words: state, upper bits, rays above, T_ref bits, any exempt
constexpr int SEL_STATE = 0, SEL_HIGH = 1, SEL_ABOVE = 2, SEL_T = 3, SEL_EXEMPT = 4, SEL_W = 8;
constexpr uint32_t SEL_OFF = 0, SEL_PASS2 = 1, SEL_DONE = 2;
constexpr int WBITS = 28;                    // merge weights below 2^28
constexpr uint32_t NO_GROUP = 0xffffffffu;   // a queue slot that is in no group
constexpr int GSUMS = 6;                     // integer sums: weight, weighted x, y, z, distance, level
constexpr int LEAD_SLAB = 128;               // leader-list entries a warp takes at once
constexpr uint32_t NO_LEADER = 0xffffffffu;  // an unused leader-list entry

// num / den rounded to nearest, ties to even, for num < 2^62 and a
// quotient below 2^22 (positions within a cell, distances, levels): a
// single-precision estimate (relative error below 2^-22, so under one here)
// corrected to the exact floor by the integer remainder, without a 64-bit
// integer division or the FP64 pipe
__device__ __forceinline__ unsigned long long div_rne(unsigned long long num, unsigned long long den) {
    unsigned long long q = (unsigned long long)__fdiv_rn((float)num, (float)den);
    long long r = (long long)(num - q * den);
    if (r < 0) { --q; r += (long long)den; }
    if (r < 0) { --q; r += (long long)den; }
    if (r >= (long long)den) { ++q; r -= (long long)den; }
    if (r >= (long long)den) { ++q; r -= (long long)den; }
    if (2 * (unsigned long long)r > den || (2 * (unsigned long long)r == den && (q & 1ull))) ++q;
    return q;
}

// does simulation `sim` merge at the end of this step
__device__ __forceinline__ bool merges(const SimDev &S, const SimAcc &a) {
    return S.active && S.merge && a.p_rays_out > (double)S.k_ex;
}

// warp-aggregated histogram increment; bin < 0: nothing
__device__ __forceinline__ void hist_add(uint32_t *hist, long long bin) {
    const unsigned peers = __match_any_sync(FULL, bin);
    const int lane = lane_id();
    if (bin >= 0 && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(hist + bin, (uint32_t)__popc(peers));
}

// the simulation a queued ray belongs to
__device__ __forceinline__ int ray_sim(const Queue &q, const Emitters &em, long long i, uint32_t e) {
    return (e & MERGED_BIT) ? (int)((q.ma[i] >> 16) & 0x7fffu) : __ldg(&em.cell[e]).w;
}

// The contiguous queue slots [c0, c1) a warp owns in the group pass (the
// march writes a parent's children next to each other: one warp sees them
// together and combines their group sums).
__device__ __forceinline__ long long warp_chunk_len(long long n, long long nwarps) {
    return ((n + 31) / 32 + nwarps - 1) / nwarps * 32;
}
__device__ __forceinline__ void warp_chunk(long long n, long long &c0, long long &c1) {
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long per = warp_chunk_len(n, nw);
    c0 = min(w * per, n);
    c1 = min(c0 + per, n);
}

// inclusive scan of one value per thread over a block of 1024 threads
__device__ unsigned long long block_incl_scan(unsigned long long v, unsigned long long *sh) {
    const int lane = lane_id(), wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += t;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const unsigned long long r = v + (wid > 0 ? sh[wid - 1] : 0ull);
    __syncthreads();
    return r;
}

// In hist[0..HIST_BINS) find the largest bin b with above + count(bins >= b)
// >= K (K > above, and the total reaches K).  Returns b and the count above b.
__device__ void select_bin(const uint32_t *hist, unsigned long long above, unsigned long long K, uint32_t *out_bin,
                           unsigned long long *out_above, unsigned long long *sh) {
    constexpr int PER = HIST_BINS / 1024;
    const int t = threadIdx.x;
    const int chunk = 1023 - t;           // thread 0 owns the highest bins
    unsigned long long v = 0;
    for (int k = 0; k < PER; ++k) v += hist[chunk * PER + k];
    const unsigned long long incl = above + block_incl_scan(v, sh);
    const unsigned long long excl = incl - v;
    if (excl < K && K <= incl) {
        unsigned long long acc = excl;
        for (int k = PER - 1; k >= 0; --k) {
            const unsigned long long c = hist[chunk * PER + k];
            if (acc + c >= K) {
                *out_bin = (uint32_t)(chunk * PER + k);
                *out_above = acc;
                break;
            }
            acc += c;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// merge-sphere rotations of the cells of merging simulations
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mrot(MergeArgs A) {
    extern __shared__ long long sh_rng[];
    long long *s_pref = sh_rng, *s_cell0 = sh_rng + A.nsims + 1;
    int *s_sim = reinterpret_cast<int *>(s_cell0 + A.nsims);
    const Ctl *C = A.ctl;
    const int nrng = C->n_ranges;
    for (int i = threadIdx.x; i <= nrng; i += blockDim.x) s_pref[i] = A.rg.pref[i];
    for (int i = threadIdx.x; i < nrng; i += blockDim.x) { s_cell0[i] = A.rg.cell0[i]; s_sim[i] = A.rg.sim[i]; }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctl->mlead = 0ull;
    if (C->err) return;
    const long long n = C->ncell_active;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nrng;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_pref[mid] <= i) lo = mid; else hi = mid;
        }
        const int sim = s_sim[lo];
        const SimDev &S = A.sims[sim];
        if (!merges(S, A.acc[sim])) continue;
        const long long local = i - s_pref[lo];
        int4 rows[3];
        rotation_rows(S.seed, (1LL << 31) + local, S.step, S.rotate, rows);
        int4 *dst = A.w.rot + 3 * (s_cell0[lo] + local);
        dst[0] = rows[0]; dst[1] = rows[1]; dst[2] = rows[2];
    }
}

// ---------------------------------------------------------------------------
// rank contents and the first histogram
// ---------------------------------------------------------------------------
// the histogram copy a block adds to (copies spread the atomics on hot bins)
__device__ __forceinline__ long long hist_row(const MergeWork &w, int sim) {
    return ((long long)sim * w.hrep + (long long)(blockIdx.x % w.hrep)) * HIST_BINS;
}

__global__ void __launch_bounds__(256) k_mhist1(MergeArgs A) {
    const Ctl *C = A.ctl;
    if (C->err) return;
    const int par = C->par;
    const Queue q = A.q[par ^ 1];
    const long long n = C->cnt[par ^ 1];
    const long long nr = (n + 31) & ~31LL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x) {
        long long bin = -1;
        if (i < n) {
            int sim = -1;
            uint32_t key = 0;
            const uint32_t pl = q.pl[i];
            if (pl != DEAD_RAY) {
                const uint32_t e = q.em[i];
                const int s = ray_sim(q, A.em, i, e);
                const SimDev &S = A.sims[s];
                if (merges(S, A.acc[s])) {
                    float T = 0.0f;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b)
                        if (b < S.nb) T += q.ph[b][i];
                    key = __float_as_uint(T);
                    sim = s;
                    bin = hist_row(A.w, s) + (key >> 16);
                }
            }
            A.w.tkey[i] = key;
            A.w.tsim[i] = sim;
        }
        hist_add(A.w.hist, bin);
    }
}

// sum each simulation's histogram copies into copy 0 (and clear the others)
__global__ void __launch_bounds__(256) k_mreduce(MergeArgs A, int pass) {
    const Ctl *C = A.ctl;
    if (C->err) return;
    const int hrep = A.w.hrep;
    const long long n = (long long)A.nsims * HIST_BINS;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / HIST_BINS);
        const bool on = pass == 1 ? merges(A.sims[s], A.acc[s]) : A.w.sel[SEL_W * s + SEL_STATE] == SEL_PASS2;
        if (!on) continue;
        uint32_t *h = A.w.hist + (long long)s * hrep * HIST_BINS + (i % HIST_BINS);
        // every copy's count first (independent loads in flight together),
        // then the clears
        uint32_t cnt[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) cnt[c] = c < hrep ? h[(long long)c * HIST_BINS] : 0u;
        uint32_t sum = 0u;
#pragma unroll
        for (int c = 0; c < 32; ++c) sum += cnt[c];
        for (int c = 1; c < hrep; ++c) h[(long long)c * HIST_BINS] = 0u;
        h[0] = sum;
    }
}

// ---------------------------------------------------------------------------
// per simulation: the threshold's upper 16 bits (pass 1) or all 32 (pass 2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_mfind(MergeArgs A, int pass) {
    __shared__ unsigned long long sh[32];
    __shared__ uint32_t s_bin;
    __shared__ unsigned long long s_above;
    Ctl *C = A.ctl;
    const int s = blockIdx.x;
    if (C->err) return;
    uint32_t *sel = A.w.sel + SEL_W * s;
    uint32_t *hist = A.w.hist + (long long)s * A.w.hrep * HIST_BINS;
    const SimDev &S = A.sims[s];
    if (pass == 1) {
        if (!merges(S, A.acc[s])) {
            if (threadIdx.x == 0) sel[SEL_STATE] = SEL_OFF;
            return;
        }
        if (threadIdx.x == 0) C->merged = 1;
        const unsigned long long K = S.k_ex > 0 ? (unsigned long long)S.k_ex : 1ull;
        select_bin(hist, 0ull, K, &s_bin, &s_above, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            sel[SEL_STATE] = SEL_PASS2;
            sel[SEL_HIGH] = s_bin;
            sel[SEL_ABOVE] = (uint32_t)s_above;
            sel[SEL_EXEMPT] = S.k_ex > 0 ? 1u : 0u;
        }
    } else {
        if (sel[SEL_STATE] != SEL_PASS2) return;
        const unsigned long long K = S.k_ex > 0 ? (unsigned long long)S.k_ex : 1ull;
        select_bin(hist, (unsigned long long)sel[SEL_ABOVE], K, &s_bin, &s_above, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            sel[SEL_T] = (sel[SEL_HIGH] << 16) | s_bin;
            sel[SEL_STATE] = SEL_DONE;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < HIST_BINS; k += blockDim.x) hist[k] = 0u;   // ready for the next pass
}

__global__ void __launch_bounds__(256) k_mhist2(MergeArgs A) {
    const Ctl *C = A.ctl;
    if (C->err) return;
    const int par = C->par;
    const long long n = C->cnt[par ^ 1];
    const long long nr = (n + 31) & ~31LL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x) {
        long long bin = -1;
        if (i < n) {
            const int sim = A.w.tsim[i];
            if (sim >= 0) {
                const uint32_t *sel = A.w.sel + SEL_W * sim;
                const uint32_t key = A.w.tkey[i];
                if (sel[SEL_STATE] == SEL_PASS2 && (key >> 16) == sel[SEL_HIGH])
                    bin = hist_row(A.w, sim) + (key & 0xffffu);
            }
        }
        hist_add(A.w.hist, bin);
    }
}

// ---------------------------------------------------------------------------
// groups: end cell and merge pixel of every non-exempt ray
// ---------------------------------------------------------------------------
// Sums of equal groups are combined within the warp first (the march writes
// a parent's split children next to each other, and they usually share cell
// and pixel).  Exempt rays are decided from two words and left untouched;
// a non-exempt ray's words are all loaded before its emitter and the cell's
// rotation, which depend on them.
__global__ void __launch_bounds__(256, 4) k_mgroup(MergeArgs A) {
    Ctl *C = A.ctl;
    if (C->err || !C->merged) return;
    const int par = C->par;
    const Queue q = A.q[par ^ 1];
    const long long n = C->cnt[par ^ 1];
    const int ndir = A.w.ndir, gw = A.w.grp_w;
    const int lane = lane_id();
    // this warp's run of leader-list entries [lslab, lslab + lleft), taken
    // LEAD_SLAB at a time with one atomic (a single shared counter per warp
    // iteration serialises the kernel)
    unsigned long long lslab = 0;
    int lleft = 0;
    long long c0, c1;
    warp_chunk(n, c0, c1);
    for (long long base = c0; base < c1; base += 32) {
        const long long i = base + lane;
        long long slot = -1;
        uint4 pack = make_uint4(NO_GROUP, 0u, 0u, 0u);
        float f[MAXB + 4];
#pragma unroll
        for (int k = 0; k < MAXB + 4; ++k) f[k] = 0.0f;
        int nbf = 0;
        int sim = -1;
        uint32_t key = 0;
        if (i < c1) {
            sim = A.w.tsim[i];
            key = A.w.tkey[i];
        }
        if (sim >= 0) {
            const uint32_t *sel = A.w.sel + SEL_W * sim;
            const uint32_t tref = sel[SEL_T];
            if (sel[SEL_STATE] == SEL_DONE && !(sel[SEL_EXEMPT] && key >= tref)) {
                const SimDev &S = A.sims[sim];
                const uint32_t e = q.em[i], pl = q.pl[i];
                const int bi = q.bi[i];
                const int dx = q.dx[i], dy = q.dy[i], dz = q.dz[i];
                const int nbs = S.nb;
#pragma unroll
                for (int b = 0; b < MAXB; ++b)
                    if (b < nbs) f[b] = q.ph[b][i];
                const int lev = (int)(pl >> LEVEL_SHIFT);
                // end point of this step's march and the distance travelled
                long long p[3];
                int dist;
                float thr;
                if (e & MERGED_BIT) {
                    const long long k = S.step - bi;
                    p[0] = q.mx[i] + k * dx; p[1] = q.my[i] + k * dy; p[2] = q.mz[i] + k * dz;
                    dist = (int)(q.ma[i] & 0xffffu) + (int)k;
                    thr = q.mthr[i];
                } else {
                    const int4 ec = __ldg(&A.em.cell[e]);
                    const long long k = S.step - bi + 1;
                    p[0] = ((2LL * ec.x + 1) << (FRAC_BITS - 1)) + k * dx;
                    p[1] = ((2LL * ec.y + 1) << (FRAC_BITS - 1)) + k * dy;
                    p[2] = ((2LL * ec.z + 1) << (FRAC_BITS - 1)) + k * dz;
                    dist = (int)k;
                    thr = S.eps_term * __ldg(&A.em.n0[e]) * pow2_neg(2 * (lev - S.l_src));
                }
                const long long cx = p[0] >> FRAC_BITS, cy = p[1] >> FRAC_BITS, cz = p[2] >> FRAC_BITS;
                if (cx >= 0 && cy >= 0 && cz >= 0 && cx < S.nx && cy < S.ny && cz < S.nz) {
                    const long long g = S.cell_off + (cz * S.ny + cy) * S.nx + cx;
                    const int4 *rp = A.w.rot + 3 * g;
                    const int4 rows[3] = {rp[0], rp[1], rp[2]};
                    slot = g * ndir + merge_pixel(S.l_merge, rows, dx, dy, dz);
                    // the end point's offsets in its cell (21 bits each), the
                    // distance (16 bits) and the level (4 bits), packed
                    const uint32_t ox = (uint32_t)(p[0] - (cx << FRAC_BITS));
                    const uint32_t oy = (uint32_t)(p[1] - (cy << FRAC_BITS));
                    const uint32_t oz = (uint32_t)(p[2] - (cz << FRAC_BITS));
                    const uint32_t ud = (uint32_t)min(dist, 65535);
                    pack = make_uint4((uint32_t)slot, ox | ((uint32_t)lev << 21), oy | ((ud & 0x7ffu) << 21),
                                      oz | ((ud >> 11) << 21));
                    nbf = nbs;
#pragma unroll
                    for (int b = 0; b <= MAXB; ++b)
                        if (b == nbs) f[b] = thr;
                }
            }
        }
        if (i < c1) A.w.tgrp[i] = pack;
        // combine equal groups in the warp, then one set of atomics per group
        const unsigned peers = __match_any_sync(FULL, slot);
        const unsigned below = peers & ((1u << lane) - 1u);
        if (__any_sync(FULL, slot >= 0 && __popc(peers) > 1)) peer_sum<MAXB + 4, float>(peers, f);
        const uint32_t kmax = __reduce_max_sync(peers, slot >= 0 ? key : 0u);
        bool leads = false;
        if (slot >= 0) {
            uint32_t gbase = 0;
            if (below == 0u) {
                gbase = atomicAdd(A.w.gcnt + slot, (uint32_t)__popc(peers));
                atomicMax(A.w.gmax + slot, kmax);
                float4 *gf = reinterpret_cast<float4 *>(A.w.grp + slot * gw + 2 * GSUMS);
#pragma unroll
                for (int b = 0; b <= MAXB; b += 4)
                    if (b <= nbf) red_add_v4(gf + b / 4, f[b], f[b + 1], f[b + 2], f[b + 3]);
            }
            // the group's first member in arrival order leads it; the
            // others leave the queue
            const int lead = __ffs(peers) - 1;
            gbase = __shfl_sync(peers, gbase, lead);
            const uint32_t rank = gbase + (uint32_t)__popc(below);
            leads = rank == 0u;
            if (!leads) q.pl[i] = DEAD_RAY;
        }
        // list the leaders: the rest of the warp's run first, then a new run
        const unsigned lm = __ballot_sync(FULL, leads);
        const int tot = __popc(lm);
        if (tot) {
            const unsigned long long s0 = lslab;
            const int left = lleft;
            unsigned long long s1 = 0;
            if (tot > left) {
                const int need = tot - left;
                const int want = need > LEAD_SLAB ? need : LEAD_SLAB;
                unsigned long long nb = 0;
                if (lane == 0) nb = atomicAdd(&C->mlead, (unsigned long long)want);
                nb = __shfl_sync(FULL, nb, 0);
                s1 = nb;
                lslab = nb + need;
                lleft = want - need;
            } else {
                lslab = s0 + tot;
                lleft = left - tot;
            }
            if (leads) {
                const int k = __popc(lm & ((1u << lane) - 1u));
                const unsigned long long o = k < left ? s0 + k : s1 + (k - left);
                if (o < (unsigned long long)A.w.lead_cap) {
                    A.w.lead_i[o] = (uint32_t)i;
                    A.w.lead_slot[o] = (uint32_t)slot;
                } else {
                    atomicOr(&C->err, 1);
                }
            }
        }
    }
    // the unused end of the warp's run
    for (int k = lane; k < lleft; k += 32)
        if (lslab + k < (unsigned long long)A.w.lead_cap) A.w.lead_i[lslab + k] = NO_LEADER;
}

// ---------------------------------------------------------------------------
// photon-weighted sums of the grouped rays
// ---------------------------------------------------------------------------
// A ray's weight is its content scaled by 2^(28 - e), where 2^e is the power
// of two above its group's largest content (exact power-of-two scaling),
// truncated and at least 1: the brightest member has at least 27 significant
// bits, every weight is below 2^28.  Weighted sums are 64-bit integers.
__global__ void __launch_bounds__(256, 4) k_mweight(MergeArgs A) {
    const Ctl *C = A.ctl;
    if (C->err || !C->merged) return;
    const long long n = C->cnt[C->par ^ 1];
    const int gw = A.w.grp_w;
    const int lane = lane_id();
    long long c0, c1;
    warp_chunk(n, c0, c1);
    for (long long base = c0; base < c1; base += 32) {
        const long long i = base + lane;
        uint4 pk = make_uint4(NO_GROUP, 0u, 0u, 0u);
        uint32_t key = 0;
        if (i < c1) {
            pk = A.w.tgrp[i];
            if (pk.x != NO_GROUP) key = A.w.tkey[i];
        }
        long long slot = pk.x == NO_GROUP ? -1 : (long long)pk.x;
        // a ray alone in its group stays as it is: its sums are never read
        if (slot >= 0 && A.w.gcnt[slot] < 2u) slot = -1;
        unsigned long long v[GSUMS] = {0, 0, 0, 0, 0, 0};
        if (slot >= 0) {
            const uint32_t gm = A.w.gmax[slot];
            const int eb = max((int)((gm >> 23) & 0xffu), 30);      // biased exponent; 2^(eb-126) > content
            const float wscale = __int_as_float((253 + WBITS - eb) << 23);
            const unsigned long long qw = max(__float2ull_rz(__fmul_rn(__uint_as_float(key), wscale)), 1ull);
            v[0] = qw;
            v[1] = qw * (unsigned long long)(pk.y & 0x1fffffu);
            v[2] = qw * (unsigned long long)(pk.z & 0x1fffffu);
            v[3] = qw * (unsigned long long)(pk.w & 0x1fffffu);
            v[4] = qw * (unsigned long long)((pk.z >> 21) | ((pk.w >> 21) << 11));
            v[5] = qw * (unsigned long long)(pk.y >> 21);
        }
        const unsigned peers = __match_any_sync(FULL, slot);
        if (__any_sync(FULL, slot >= 0 && __popc(peers) > 1)) peer_sum<GSUMS, unsigned long long>(peers, v);
        if (slot >= 0 && (peers & ((1u << lane) - 1u)) == 0u) {
            unsigned long long *gs = reinterpret_cast<unsigned long long *>(A.w.grp + slot * gw);
#pragma unroll
            for (int k = 0; k < GSUMS; ++k) atomicAdd(gs + k, v[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// in place: merged rays into their leaders' slots
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_memit(MergeArgs A) {
    extern __shared__ int sh_drop[];              // per simulation: rays removed by merging
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x) sh_drop[k] = 0;
    __syncthreads();
    const Ctl *C = A.ctl;
    if (!C->err && C->merged) {
        const Queue q = A.q[C->par ^ 1];
        const long long nl = min((long long)C->mlead, A.w.lead_cap);
        const int ndir = A.w.ndir, gw = A.w.grp_w, nbq = A.nbq;
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nl;
             k += (long long)gridDim.x * blockDim.x) {
            const uint32_t li = A.w.lead_i[k];
            if (li == NO_LEADER) continue;
            const long long i = li;
            const uint32_t slot = A.w.lead_slot[k];
            const uint32_t gsize = A.w.gcnt[slot];
            if (gsize > 1) {
                const int sim = A.w.tsim[i];
                const SimDev &S = A.sims[sim];
                const float *gp = A.w.grp + (long long)slot * gw;
                const unsigned long long *gs = reinterpret_cast<const unsigned long long *>(gp);
                const unsigned long long W = gs[0];
                // weights below 2^28 and offsets below 2^21: the sums stay
                // exact while W < 2^41 (more than 2^13 members as bright as
                // the brightest would be needed to reach it)
                if (W >= (1ull << 41)) atomicOr((int *)&C->err, 8);
                const long long g = (long long)slot / ndir;
                const uint32_t pm = slot % ndir;
                const int local = (int)(g - S.cell_off);          // below 2^31 cells
                const int cell[3] = {local % S.nx, (local / S.nx) % S.ny, local / (S.nx * S.ny)};
                int P[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) P[a] = (cell[a] << FRAC_BITS) + (int)div_rne(gs[1 + a], W);
                const int Adist = (int)min(div_rne(gs[4], W), 65535ull);
                const int L2 = min(max((int)div_rne(gs[5], W), S.l_merge), S.l_max);
                const float *gph = gp + 2 * GSUMS;
                const int4 *rp = A.w.rot + 3 * g;
                const int4 rows[3] = {rp[0], rp[1], rp[2]};
                const int4 vq = S.l_merge <= A.ltab ? __ldg(&A.pixtab[level_offset(S.l_merge) + pm])
                                                    : healpix_vq(S.l_merge, pm);
                int32_t dx, dy, dz;
                rotate_dir(rows, vq, dx, dy, dz);
                q.pl[i] = ((uint32_t)L2 << LEVEL_SHIFT) | pm;
                q.em[i] = MERGED_BIT | (uint32_t)local;
                q.bi[i] = S.step;
                q.dx[i] = dx; q.dy[i] = dy; q.dz[i] = dz;
#pragma unroll
                for (int b = 0; b < MAXB; ++b)
                    if (b < nbq) q.ph[b][i] = b < S.nb ? gph[b] : 0.0f;
                q.mx[i] = P[0]; q.my[i] = P[1]; q.mz[i] = P[2];
                q.ma[i] = (L2 > S.l_merge ? 0x80000000u : 0u) | ((uint32_t)sim << 16) | (uint32_t)Adist;
                q.mthr[i] = gph[S.nb];
                atomicAdd(&sh_drop[sim], (int)gsize - 1);
            }
            // the leader clears its group for the next step
            float4 *gz = reinterpret_cast<float4 *>(A.w.grp + (long long)slot * gw);
            for (int b = 0; b < gw / 4; ++b) gz[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            A.w.gcnt[slot] = 0u;
            A.w.gmax[slot] = 0u;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x)
        if (sh_drop[k]) atomicAdd(&A.acc[k].p_rays_out, -(double)sh_drop[k]);
}

__global__ void k_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, int per_ray,
                                    uint32_t *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int32_t *R = Rq + (per_ray ? 9 * i : 0);
        int4 rows[3];
        for (int k = 0; k < 3; ++k) rows[k] = make_int4(R[3 * k], R[3 * k + 1], R[3 * k + 2], 0);
        out[i] = merge_pixel(level, rows, d[3 * i], d[3 * i + 1], d[3 * i + 2]);
    }
}

cudaError_t launch_merge(const MergeArgs &a, int sm_count, cudaStream_t st) {
    const int rblocks = std::min(sm_count * 16, MERGE_MAX_BLOCKS);
    const size_t rng_sh = (size_t)(2 * a.nsims + 1) * sizeof(long long) + (size_t)a.nsims * sizeof(int);
    k_mrot<<<rblocks, 256, rng_sh, st>>>(a);
    k_mhist1<<<rblocks, 256, 0, st>>>(a);
    if (a.w.hrep > 1) k_mreduce<<<rblocks, 256, 0, st>>>(a, 1);
    k_mfind<<<a.nsims, 1024, 0, st>>>(a, 1);
    k_mhist2<<<rblocks, 256, 0, st>>>(a);
    if (a.w.hrep > 1) k_mreduce<<<rblocks, 256, 0, st>>>(a, 2);
    k_mfind<<<a.nsims, 1024, 0, st>>>(a, 2);
    k_mgroup<<<rblocks, 256, 0, st>>>(a);
    k_mweight<<<rblocks, 256, 0, st>>>(a);
    k_memit<<<rblocks, 256, (size_t)a.nsims * sizeof(int), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, bool per_ray,
                                     uint32_t *out, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_probe_merge_pixel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(level, n, d, Rq, per_ray ? 1 : 0, out);
    return cudaGetLastError();
}

}  // namespace frt
