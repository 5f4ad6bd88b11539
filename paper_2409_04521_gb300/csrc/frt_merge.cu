// frt_merge.cu -- ray merging at the end of a step (Sec. 3.3, Eq. 4) and the
// march variants that carry merged rays.
//
// The step, per simulation that merges (it has more live rays than
// K = floor(N_ex * N_RT)):
//   k_mrot   : per cell, the random rotation of the cell's merge sphere for
//              this step (key 2^31 + local cell index);
//   k_mhist1 : per ray, its content (single-precision sum of its bins, the
//              quantity ranked) and a histogram of the content's upper 16 bits;
//   k_mfind  : per simulation, a two-pass radix select of the K-th largest
//              content T_ref (the largest when K = 0): with K > 0 every ray
//              at least that bright is exempt;
//   k_mhist2 : per ray in the selected upper bin, a histogram of the lower bits;
//   k_mgroup : per non-exempt ray, its end cell and merge pixel; a group slot
//              per (cell, pixel) takes its photons and threshold (vector
//              reductions), its weighted position, distance and level as
//              exact 64-bit integer sums, and the ray's arrival rank (rank 0
//              leads the group).  The weight is the content on a grid of
//              2^-26 of the power of two above T_ref (at least 1), so the
//              means are exact quotients, independent of summation order;
//   k_mscan  : the new queue length L (rays left: exempt, lone, one per group)
//              and the number H of holes below it;
//   k_memit  : in place: each group's leader overwrites its own slot with the
//              merged ray and clears the group; holes below L and live rays
//              at or above L are listed;
//   k_mmove  : the H live rays at or above L move down into the H holes.
// Contents are non-negative floats, so their bit patterns order as unsigned
// integers and the select works on the bits.
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
constexpr int WBITS = 26;                    // merge weights below 2^26
constexpr int GSUMS = 6;                     // integer sums: weight, weighted x, y, z, distance, level

// num / den rounded to nearest, ties to even
__device__ __forceinline__ unsigned long long div_rne(unsigned long long num, unsigned long long den) {
    unsigned long long q = num / den, r = num - q * den;
    if (2 * r > den || (2 * r == den && (q & 1ull))) ++q;
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

// The contiguous queue slots [c0, c1) a warp owns in the group and emit
// passes (the same for both, so per-warp prefix counts follow slot order).
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

// a ray that stays live after the merge: exempt, alone in its group, or a leader
__device__ __forceinline__ bool stays(uint32_t pl, uint32_t gid) {
    return pl != DEAD_RAY && (gid == MERGE_KEEP || !(gid & MERGE_FOLLOWER));
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
        merge_rotation_rows(S.seed, local, S.step, S.rotate, rows);
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
        uint32_t sum = h[0];
        for (int c = 1; c < hrep; ++c) {
            sum += h[(long long)c * HIST_BINS];
            h[(long long)c * HIST_BINS] = 0u;
        }
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
// and pixel).  Every ray's fate is known here -- exempt, lone and group
// leaders go to the merged queue, followers do not -- so the pass also
// counts each warp's outputs for the exact compaction of k_memit (both
// kernels give a warp the same queue slots).
__global__ void __launch_bounds__(256, 5) k_mgroup(MergeArgs A) {
    const Ctl *C = A.ctl;
    const bool on = !C->err && C->merged;
    uint32_t outs = 0;
    if (on) {
        const int par = C->par;
        const Queue q = A.q[par ^ 1];
        const long long n = C->cnt[par ^ 1];
        const int ndir = A.w.ndir, gw = A.w.grp_w;
        const int lane = lane_id();
        long long c0, c1;
        warp_chunk(n, c0, c1);
        for (long long base = c0; base < c1; base += 32) {
            const long long i = base + lane;
            uint32_t gid = MERGE_KEEP;
            long long slot = -1;
            unsigned long long v[GSUMS] = {0, 0, 0, 0, 0, 0};
            float f[MAXB + 4];
#pragma unroll
            for (int k = 0; k < MAXB + 4; ++k) f[k] = 0.0f;
            int nbf = 0;
            bool live = false;
            if (i < c1) {
                live = q.pl[i] != DEAD_RAY;
                const int sim = A.w.tsim[i];
                if (sim >= 0) {
                    const uint32_t *sel = A.w.sel + SEL_W * sim;
                    const uint32_t key = A.w.tkey[i];
                    const uint32_t tref = sel[SEL_T];
                    if (sel[SEL_STATE] == SEL_DONE && !(sel[SEL_EXEMPT] && key >= tref)) {
                        const SimDev &S = A.sims[sim];
                        const uint32_t e = q.em[i], pl = q.pl[i];
                        const int bi = q.bi[i];
                        const int dx = q.dx[i], dy = q.dy[i], dz = q.dz[i];
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
                            // weight: the content times 2^(26 - e), T_ref < 2^e
                            // (exact power-of-two scaling), truncated, at least 1
                            const int eref = (int)((tref >> 23) & 0xffu) - 126;
                            const float wscale = __int_as_float((127 + WBITS - eref) << 23);
                            const unsigned long long qw =
                                max(__float2ull_rz(__fmul_rn(__uint_as_float(key), wscale)), 1ull);
                            v[0] = qw;
                            v[1] = qw * (unsigned long long)(p[0] - (cx << FRAC_BITS));
                            v[2] = qw * (unsigned long long)(p[1] - (cy << FRAC_BITS));
                            v[3] = qw * (unsigned long long)(p[2] - (cz << FRAC_BITS));
                            v[4] = qw * (unsigned long long)dist;
                            v[5] = qw * (unsigned long long)lev;
                            nbf = S.nb;
#pragma unroll
                            for (int b = 0; b < MAXB; ++b) {
                                if (b < S.nb) f[b] = q.ph[b][i];
                                if (b == S.nb) f[b] = thr;
                            }
                            if (S.nb == MAXB) f[MAXB] = thr;
                        }
                    }
                }
            }
            // combine equal groups in the warp, then one set of atomics per group
            const unsigned peers = __match_any_sync(FULL, slot);
            const unsigned below = peers & ((1u << lane) - 1u);
            if (__any_sync(FULL, slot >= 0 && __popc(peers) > 1)) {
                peer_sum<GSUMS, unsigned long long>(peers, v);
                peer_sum<MAXB + 4, float>(peers, f);
            }
            if (slot >= 0) {
                uint32_t base = 0;
                if (below == 0u) {
                    base = atomicAdd(A.w.gcnt + slot, (uint32_t)__popc(peers));
                    float *gp = A.w.grp + slot * gw;
                    unsigned long long *gs = reinterpret_cast<unsigned long long *>(gp);
                    for (int k = 0; k < GSUMS; ++k) atomicAdd(gs + k, v[k]);
                    float4 *gf = reinterpret_cast<float4 *>(gp + 2 * GSUMS);
#pragma unroll
                    for (int b = 0; b <= MAXB; b += 4)
                        if (b <= nbf) red_add_v4(gf + b / 4, f[b], f[b + 1], f[b + 2], f[b + 3]);
                }
                // the group's first member in arrival order leads it
                const int lead = __ffs(peers) - 1;
                base = __shfl_sync(peers, base, lead);
                const uint32_t rank = base + (uint32_t)__popc(below);
                gid = (uint32_t)slot | (rank ? MERGE_FOLLOWER : 0u);
            }
            if (i < c1) {
                A.w.gid[i] = gid;
                outs += live && (gid == MERGE_KEEP || !(gid & MERGE_FOLLOWER)) ? 1u : 0u;
            }
        }
    }
    // this warp's outputs
    uint32_t t = outs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane_id() == 0) A.w.bcount[blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)] = t;
}

// exclusive prefix of the per-warp counts of rays that stay; the new queue
// length L and the number H of holes below it
__global__ void __launch_bounds__(1024) k_mscan(MergeArgs A, int nwarps) {
    __shared__ unsigned long long sh[32];
    Ctl *C = A.ctl;
    if (C->err || !C->merged) return;
    unsigned long long run = 0;
    for (int b0 = 0; b0 < nwarps; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const unsigned long long v = b < nwarps ? A.w.bcount[b] : 0ull;
        const unsigned long long incl = block_incl_scan(v, sh);
        if (b < nwarps) A.w.boff[b] = (long long)(run + incl - v);
        if (threadIdx.x == blockDim.x - 1) sh[0] = incl;     // block_incl_scan's last barrier has passed
        __syncthreads();
        run += sh[0];
        __syncthreads();
    }
    // rays that stay below L: the prefix of L's warp plus its own below L
    const int par = C->par;
    const long long n = C->cnt[par ^ 1];
    const long long L = (long long)run;
    const long long per = warp_chunk_len(n, nwarps);
    unsigned long long below = 0;
    if (L < n) {
        const long long w = L / per;
        const Queue q = A.q[par ^ 1];
        unsigned long long c = 0;
        for (long long i = w * per + threadIdx.x; i < L; i += blockDim.x) c += stays(q.pl[i], A.w.gid[i]) ? 1ull : 0ull;
        const unsigned long long tot = block_incl_scan(c, sh);
        if (threadIdx.x == blockDim.x - 1) sh[0] = tot;
        __syncthreads();
        below = (unsigned long long)A.w.boff[w] + sh[0];
    } else {
        below = run;
    }
    if (threadIdx.x == 0) {
        C->mlive = L;
        C->mmoves = L - (long long)below;
    }
}

// ---------------------------------------------------------------------------
// in place: merged rays into their leaders' slots; holes and movers listed
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_memit(MergeArgs A) {
    extern __shared__ int sh_drop[];              // per simulation: rays removed by merging
    __shared__ int s_done;                        // warps of this block that have finished
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x) sh_drop[k] = 0;
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    Ctl *C = A.ctl;
    if (!C->err && C->merged) {
        const int par = C->par;
        const Queue q = A.q[par ^ 1];
        const long long n = C->cnt[par ^ 1];
        const long long L = C->mlive;
        const int ndir = A.w.ndir, gw = A.w.grp_w, nbq = A.nbq;
        const int lane = lane_id();
        long long c0, c1;
        warp_chunk(n, c0, c1);
        long long rank0 = A.w.boff[blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)];
        for (long long base = c0; base < c1; base += 32) {
            const long long i = base + lane;
            bool stay = false, leader = false;
            uint32_t slot = 0, gsize = 0;
            if (i < c1) {
                const uint32_t pl = q.pl[i], gid = A.w.gid[i];
                stay = stays(pl, gid);
                if (stay && gid != MERGE_KEEP) {
                    leader = true;
                    slot = gid;
                    gsize = A.w.gcnt[slot];
                }
            }
            const unsigned has = __ballot_sync(FULL, stay);
            const long long rank = rank0 + __popc(has & ((1u << lane) - 1u));   // live rays before slot i
            rank0 += __popc(has);
            if (i < c1) {
                if (!stay && i < L) A.w.hole[i - rank] = (uint32_t)i;
                if (stay && i >= L) A.w.mover[L - 1 - rank] = (uint32_t)i;
            }
            if (leader && gsize > 1) {
                const int sim = A.w.tsim[i];
                const SimDev &S = A.sims[sim];
                const float *gp = A.w.grp + (long long)slot * gw;
                const unsigned long long *gs = reinterpret_cast<const unsigned long long *>(gp);
                const unsigned long long W = gs[0];
                const long long g = (long long)slot / ndir;
                const uint32_t pm = slot % ndir;
                const long long local = g - S.cell_off;
                const long long cell[3] = {local % S.nx, (local / S.nx) % S.ny, local / ((long long)S.nx * S.ny)};
                int P[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) P[k] = (int)(cell[k] << FRAC_BITS) + (int)div_rne(gs[1 + k], W);
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
                for (int k = 0; k < MAXB; ++k)
                    if (k < nbq) q.ph[k][i] = k < S.nb ? gph[k] : 0.0f;
                q.mx[i] = P[0]; q.my[i] = P[1]; q.mz[i] = P[2];
                q.ma[i] = (L2 > S.l_merge ? 0x80000000u : 0u) | ((uint32_t)sim << 16) | (uint32_t)Adist;
                q.mthr[i] = gph[S.nb];
                atomicAdd(&sh_drop[sim], (int)gsize - 1);
            }
            if (leader) {
                // the leader clears its group for the next step
                float4 *gz = reinterpret_cast<float4 *>(A.w.grp + (long long)slot * gw);
                for (int k = 0; k < gw / 4; ++k) gz[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                A.w.gcnt[slot] = 0u;
            }
        }
    }
    // the block's last warp to finish adds the block's counts (no barrier:
    // warps of unequal work do not wait for each other)
    __threadfence_block();
    int last = 0;
    if (lane_id() == 0) last = atomicAdd(&s_done, 1) == (int)(blockDim.x >> 5) - 1;
    last = __shfl_sync(FULL, last, 0);
    if (last) {
        __threadfence_block();
        for (int k = lane_id(); k < A.nsims; k += 32) {
            const int d = atomicAdd(&sh_drop[k], 0);
            if (d) atomicAdd(&A.acc[k].p_rays_out, -(double)d);
        }
    }
}

// the live rays at or above L move into the holes below it
__global__ void __launch_bounds__(256) k_mmove(MergeArgs A) {
    const Ctl *C = A.ctl;
    if (C->err || !C->merged) return;
    const Queue q = A.q[C->par ^ 1];
    const long long H = C->mmoves;
    const int nbq = A.nbq;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < H; k += (long long)gridDim.x * blockDim.x) {
        const long long i = A.w.mover[k], o = A.w.hole[k];
        const uint32_t e = q.em[i];
        q.pl[o] = q.pl[i]; q.em[o] = e; q.bi[o] = q.bi[i];
        q.dx[o] = q.dx[i]; q.dy[o] = q.dy[i]; q.dz[o] = q.dz[i];
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < nbq) q.ph[b][o] = q.ph[b][i];
        if (e & MERGED_BIT) {
            q.mx[o] = q.mx[i]; q.my[o] = q.my[i]; q.mz[o] = q.mz[i];
            q.ma[o] = q.ma[i]; q.mthr[o] = q.mthr[i];
        }
    }
}

__global__ void k_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, uint32_t *out) {
    int4 rows[3];
    for (int k = 0; k < 3; ++k) rows[k] = make_int4(Rq[3 * k], Rq[3 * k + 1], Rq[3 * k + 2], 0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = merge_pixel(level, rows, d[3 * i], d[3 * i + 1], d[3 * i + 2]);
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
    k_mscan<<<1, 1024, 0, st>>>(a, rblocks * 8);
    k_memit<<<rblocks, 256, (size_t)a.nsims * sizeof(int), st>>>(a);
    k_mmove<<<rblocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, uint32_t *out,
                                     cudaStream_t st) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_probe_merge_pixel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(level, n, d, Rq, out);
    return cudaGetLastError();
}

}  // namespace frt
