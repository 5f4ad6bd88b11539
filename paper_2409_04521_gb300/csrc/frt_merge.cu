// frt_merge.cu -- ray merging at the end of a step (Sec. 3.3, Eq. 4) and the
// march variants that carry merged rays (without Generalized Opacity mode).
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
//   k_mhist2  : per ray in the selected upper bin, a histogram of the lower
//               bits; and the candidate list, the rays that can still merge
//               (those at most in T_ref's upper bin), so that the passes
//               below run over candidates only, with whole warps;
//   k_mgroup  : per non-exempt candidate, its end cell and merge pixel; a
//               group slot per (cell, pixel) counts its members and takes the
//               largest member content and the leader (the member with the
//               lowest list index); the candidate's group slot, end point,
//               distance and level are kept per candidate;
//   k_mweight : per candidate in a group of two or more, its photons and
//               termination threshold (vector reductions; rays alone in their
//               group never load them), its photon weight --
//               the content on a grid of 2^-28 of the power of two above its
//               group's largest content, truncated, at least 1 -- and the
//               weighted end point, distance and level as exact 64-bit
//               integer sums, so the photon-weighted means are exact quotients
//               of sums that do not depend on the summation order, to 2^-27 of
//               the group's brightest member; every member leaves a hole
//               in the queue and each group's leader takes the next entry of
//               the merged-ray list; a ray alone in its group stays and
//               clears the group's word;
//   k_mscan   : the blocks' places in the appended run of merged rays;
//   k_memit   : per entry of that list, the merged ray (means rounded once),
//               appended densely after the march's output, and the group
//               cleared for the next step.
// The holes stay in the queue: the next march skips them and writes its
// survivors densely into the other queue, so no compaction pass is needed.
// Contents are non-negative floats, so their bit patterns order as unsigned
// integers and the select and the group maximum work on the bits.
#include "frt_march.cuh"

namespace frt {

// ---------------------------------------------------------------------------
// march variants with merged rays (engines without Generalized members)
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

// per-simulation selection words: state, upper bits, rays above, T_ref bits,
// any exempt, rays removed by this step's merge
constexpr int SEL_STATE = 0, SEL_HIGH = 1, SEL_ABOVE = 2, SEL_T = 3, SEL_EXEMPT = 4, SEL_DROP = 5, SEL_W = 8;
constexpr uint32_t SEL_OFF = 0, SEL_PASS2 = 1, SEL_DONE = 2;
constexpr int WBITS = 28;                    // merge weights below 2^28
constexpr uint32_t NO_GROUP = 0xffffffffu;   // a queue slot that is in no group
constexpr uint32_t NO_KEY = 0xffffffffu;     // one simulation: a slot not taking part (not a content)
constexpr int GSUMS = 6;                     // integer sums: weight, weighted x, y, z, distance, level

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
    if (!__any_sync(FULL, bin >= 0)) return;               // warp-uniform
    const unsigned peers = __match_any_sync(FULL, bin);
    const int lane = lane_id();
    if (bin >= 0 && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(hist + bin, (uint32_t)__popc(peers));
}

// the simulation a queued ray belongs to
__device__ __forceinline__ int ray_sim(const Queue &q, const Emitters &em, long long i, uint32_t e) {
    return (e & MERGED_BIT) ? (int)((q.ma[i] >> 16) & 0x7fffu) : __ldg(&em.cell[e]).w;
}

// whether a block of a pass with barriers runs: the control words are read
// once, by one thread, so that every thread of the block takes the same
// branch (another block may set the error word meanwhile)
__device__ __forceinline__ bool block_runs(const Ctl *C, bool need_merged, int *s_flag) {
    if (threadIdx.x == 0) *s_flag = C->err == 0 && (!need_merged || C->merged != 0);
    __syncthreads();
    return *s_flag != 0;
}

// inclusive prefix sum over the lanes of a warp
__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// In hist[0..HIST_BINS) find the largest bin b with above + count(bins >= b)
// >= K (K > above, and the total reaches K).  Returns b and the count above
// b.  A block of 1024 threads visits the bins from the top, d = HIST_BINS - 1
// - bin: warp w owns d in [2048 w, 2048 w + 2048), in rows of 32 bins (128
// contiguous bytes); lane l sums the rows l and l + 32 of its warp.  The warp
// holding the K-th ray then finds its row from the row sums, and the bin
// within the row.
__device__ void select_bin(const uint32_t *hist, unsigned long long above, unsigned long long K, uint32_t *out_bin,
                           unsigned long long *out_above, uint32_t (*s_rows)[64], unsigned long long *s_w) {
    constexpr int WB = HIST_BINS / 32;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t rs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int d0 = w * WB + 32 * (lane + 32 * h);
        const uint4 *src = reinterpret_cast<const uint4 *>(hist + (HIST_BINS - 32 - d0));
        uint4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = src[k];
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += v[k].x + v[k].y + v[k].z + v[k].w;
        rs[h] = t;
        s_rows[w][lane + 32 * h] = t;
    }
    unsigned long long tw = (unsigned long long)rs[0] + rs[1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tw += __shfl_xor_sync(FULL, tw, o);
    if (lane == 0) s_w[w] = tw;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = s_w[lane], inc = warp_incl_scan64(v);
        s_w[32 + lane] = inc;
        __syncwarp();
        s_w[lane] = inc - v;
    }
    __syncthreads();
    unsigned long long acc = above + s_w[w];
    if (!(acc < K && K <= above + s_w[32 + w])) return;      // warp-uniform
    int row = -1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (row >= 0) break;
        const unsigned long long v = s_rows[w][lane + 32 * h], inc = acc + warp_incl_scan64(v);
        const unsigned hit = __ballot_sync(FULL, inc - v < K && K <= inc);
        if (hit) {
            const int src = __ffs(hit) - 1;
            row = 32 * h + src;
            acc = __shfl_sync(FULL, inc - v, src);
        } else {
            acc = __shfl_sync(FULL, inc, 31);
        }
    }
    if (row < 0) return;                                     // not reached: the warp holds the K-th
    const int d = w * WB + 32 * row + lane;
    const unsigned long long c = hist[HIST_BINS - 1 - d], inc = acc + warp_incl_scan64(c);
    const unsigned hit = __ballot_sync(FULL, inc - c < K && K <= inc);
    if (lane == __ffs(hit) - 1) {
        *out_bin = (uint32_t)(HIST_BINS - 1 - d);
        *out_above = inc - c;
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
            // the ray's words together (a single simulation needs no
            // emitter lookup); bins past a member's own are zero
            const uint32_t pl = q.pl[i];
            const uint32_t e = A.nsims > 1 ? q.em[i] : 0u;
            float ph[MAXB];
#pragma unroll
            for (int b = 0; b < MAXB; ++b) ph[b] = b < A.nbq ? q.ph[b][i] : 0.0f;
            int sim = -1;
            uint32_t key = 0;
            if (pl != DEAD_RAY) {
                const int s = A.nsims > 1 ? ray_sim(q, A.em, i, e) : 0;
                if (merges(A.sims[s], A.acc[s])) {
                    float T = 0.0f;
#pragma unroll
                    for (int b = 0; b < MAXB; ++b) T += ph[b];
                    key = __float_as_uint(T);
                    sim = s;
                    bin = hist_row(A.w, s) + (key >> 16);
                }
            }
            if (A.nsims > 1) {
                A.w.tkey[i] = key;
                A.w.tsim[i] = sim;
            } else {
                A.w.tkey[i] = sim >= 0 ? key : NO_KEY;   // one simulation: the key says it all
            }
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
    __shared__ uint32_t s_rows[32][64];
    __shared__ unsigned long long s_w[64];
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
        if (threadIdx.x == 0) {
            C->merged = 1;
            s_bin = 0u;
            s_above = 0ull;
        }
        const unsigned long long K = S.k_ex > 0 ? (unsigned long long)S.k_ex : 1ull;
        select_bin(hist, 0ull, K, &s_bin, &s_above, s_rows, s_w);
        __syncthreads();
        if (threadIdx.x == 0) {
            sel[SEL_STATE] = SEL_PASS2;
            sel[SEL_HIGH] = s_bin;
            sel[SEL_ABOVE] = (uint32_t)s_above;
            sel[SEL_EXEMPT] = S.k_ex > 0 ? 1u : 0u;
        }
    } else {
        if (sel[SEL_STATE] != SEL_PASS2) return;
        if (threadIdx.x == 0) {
            s_bin = 0u;
            s_above = 0ull;
        }
        const unsigned long long K = S.k_ex > 0 ? (unsigned long long)S.k_ex : 1ull;
        select_bin(hist, (unsigned long long)sel[SEL_ABOVE], K, &s_bin, &s_above, s_rows, s_w);
        __syncthreads();
        if (threadIdx.x == 0) {
            sel[SEL_T] = (sel[SEL_HIGH] << 16) | s_bin;
            sel[SEL_STATE] = SEL_DONE;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < HIST_BINS; k += blockDim.x) hist[k] = 0u;   // ready for the next pass
}

// The candidate and merged-ray lists are built without a global counter:
// block b of the merge passes (all launched with the same grid) owns the
// queue slots [b ch, (b + 1) ch) and lists their candidates from b ch on, in
// queue order, and later its merged rays the same way; the per-block counts
// give each block's place in the queue's appended run.
__device__ __forceinline__ long long block_chunk(long long n) {
    const long long g = gridDim.x;
    return ((n + g - 1) / g + 255) & ~255LL;
}

// Exclusive positions, within a window of the block's 256 threads, of the
// threads whose flag is set; *total gets the window's count.  Two barriers:
// every thread of the block calls it, with the two buffers of s_wofs taken in
// turn by successive windows (a buffer is written again only two windows
// later, after every thread has passed the next window's barriers).
__device__ __forceinline__ uint32_t block_rank(bool flag, uint32_t *s_wofs, uint32_t *total) {
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(FULL, flag);
    if (lane == 0) s_wofs[wid] = (uint32_t)__popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < 8; ++k) {
            const uint32_t c = s_wofs[k];
            s_wofs[k] = t;
            t += c;
        }
        s_wofs[8] = t;
    }
    __syncthreads();
    const uint32_t r = s_wofs[wid] + (uint32_t)__popc(m & ((1u << lane) - 1u));
    *total = s_wofs[8];
    return r;
}

// the participating ray at slot i: its simulation (-1: none) and rank content
__device__ __forceinline__ int slot_key(const MergeArgs &A, long long i, uint32_t &key) {
    if (A.nsims > 1) {
        const int sim = A.w.tsim[i];
        key = sim >= 0 ? A.w.tkey[i] : 0u;
        return sim;
    }
    key = A.w.tkey[i];
    return key != NO_KEY ? 0 : -1;
}

// Exclusive prefix, over the block's 256 threads in order, of a per-thread
// count; *total gets the block's sum.  Two barriers, the buffers of s_wofs in
// turn as for block_rank.
__device__ __forceinline__ uint32_t block_prefix(uint32_t c, uint32_t *s_wofs, uint32_t *total) {
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_wofs[wid] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < 8; ++k) {
            const uint32_t v = s_wofs[k];
            s_wofs[k] = t;
            t += v;
        }
        s_wofs[8] = t;
    }
    __syncthreads();
    *total = s_wofs[8];
    return s_wofs[wid] + inc - c;
}

// per ray in the selected upper bin: a histogram of the lower bits; and the
// block's candidate list (the march writes a parent's children next to each
// other, and the group pass combines the sums of neighbours in the list).
// Windows of 1024 slots, four consecutive slots a thread (a single
// simulation's four keys in one 16-byte load), so that every thread has
// several loads in flight between the window's barriers.
__global__ void __launch_bounds__(256) k_mhist2(MergeArgs A) {
    __shared__ uint32_t s_wofs[2][9];
    __shared__ int s_on;
    Ctl *C = A.ctl;
    if (!block_runs(C, false, &s_on)) return;
    const int par = C->par;
    const long long n = C->cnt[par ^ 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) C->mbase = n;
    const long long ch = block_chunk(n), b0 = blockIdx.x * ch, b1 = min(n, b0 + ch);
    uint32_t run = 0;                              // candidates listed so far (block-uniform)
    int wpar = 0;
    for (long long w0 = b0; w0 < b1; w0 += 1024, wpar ^= 1) {
        const long long i0 = w0 + 4 * threadIdx.x;  // a multiple of 4: b0 is one of 256
        uint32_t key[4];
        int sim[4];
        if (A.nsims == 1 && i0 + 3 < b1) {
            const uint4 k4 = *reinterpret_cast<const uint4 *>(A.w.tkey + i0);
            key[0] = k4.x; key[1] = k4.y; key[2] = k4.z; key[3] = k4.w;
#pragma unroll
            for (int j = 0; j < 4; ++j) sim[j] = key[j] != NO_KEY ? 0 : -1;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                key[j] = 0u;
                sim[j] = i0 + j < b1 ? slot_key(A, i0 + j, key[j]) : -1;
            }
        }
        bool cand[4];
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long bin = -1;
            cand[j] = false;
            if (sim[j] >= 0) {
                const uint32_t *sel = A.w.sel + SEL_W * sim[j];
                if (sel[SEL_STATE] == SEL_PASS2) {
                    const uint32_t hi = key[j] >> 16, high = sel[SEL_HIGH];
                    if (hi == high) bin = hist_row(A.w, sim[j]) + (key[j] & 0xffffu);
                    cand[j] = !sel[SEL_EXEMPT] || hi <= high;
                }
            }
            hist_add(A.w.hist, bin);
            c += cand[j] ? 1u : 0u;
        }
        uint32_t tot;
        uint32_t r = run + block_prefix(c, s_wofs[wpar], &tot);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (cand[j]) {
                A.w.cand[b0 + r] = (uint32_t)(i0 + j);
                A.w.ckey[b0 + r] = key[j];
                ++r;
            }
        run += tot;
    }
    if (threadIdx.x == 0) A.w.bcnt[blockIdx.x] = run;
}

// ---------------------------------------------------------------------------
// groups: end cell and merge pixel of every non-exempt candidate
// ---------------------------------------------------------------------------
// Sums of equal groups are combined within the warp first (a parent's split
// children are neighbours in the list and usually share cell and pixel).
// Exempt candidates (the rays of T_ref's upper bin at least T_ref) are
// decided from two words and left untouched; a non-exempt ray's words are
// all loaded before its emitter and the cell's rotation, which depend on
// them.  Every group update is a reduction without a returned value: the
// group's leader is its member with the lowest candidate-list index (kept
// as its complement, so that a cleared group reads zero).
__global__ void __launch_bounds__(256, 4) k_mgroup(MergeArgs A) {
    Ctl *C = A.ctl;
    if (C->err || !C->merged) return;
    const int par = C->par;
    const Queue q = A.q[par ^ 1];
    const long long b0 = blockIdx.x * block_chunk(C->cnt[par ^ 1]);
    const long long b1 = b0 + A.w.bcnt[blockIdx.x];
    const int ndir = A.w.ndir;
    const int lane = lane_id();
    for (long long base = b0 + (threadIdx.x & ~31); base < b1; base += blockDim.x) {
        const long long c = base + lane;
        long long slot = -1;
        uint4 pack = make_uint4(NO_GROUP, 0u, 0u, 0u);
        int sim = -1;
        uint32_t key = 0;
        long long i = 0;
        if (c < b1) {
            i = A.w.cand[c];
            key = A.w.ckey[c];
            sim = A.nsims > 1 ? A.w.tsim[i] : 0;   // a candidate belongs to a merging simulation
        }
        if (sim >= 0) {
            const uint32_t *sel = A.w.sel + SEL_W * sim;
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
                if (e & MERGED_BIT) {
                    const long long k = S.step - bi;
                    p[0] = q.mx[i] + k * dx; p[1] = q.my[i] + k * dy; p[2] = q.mz[i] + k * dz;
                    dist = (int)(q.ma[i] & 0xffffu) + (int)k;
                } else {
                    const int4 ec = __ldg(&A.em.cell[e]);
                    const long long k = S.step - bi + 1;
                    p[0] = ((2LL * ec.x + 1) << (FRAC_BITS - 1)) + k * dx;
                    p[1] = ((2LL * ec.y + 1) << (FRAC_BITS - 1)) + k * dy;
                    p[2] = ((2LL * ec.z + 1) << (FRAC_BITS - 1)) + k * dz;
                    dist = (int)k;
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
                }
            }
        }
        if (c < b1) A.w.tgrp[c] = pack;
        // combine equal groups in the warp, then one set of reductions per group
        const unsigned peers = __match_any_sync(FULL, slot);
        const uint32_t kmax = __reduce_max_sync(peers, slot >= 0 ? key : 0u);
        if (slot >= 0 && (peers & ((1u << lane) - 1u)) == 0u) {
            uint4 *gc = A.w.gcm + slot;
            atomicAdd(&gc->x, (uint32_t)__popc(peers));
            atomicMax(&gc->y, kmax);
            atomicMax(&gc->z, ~(uint32_t)c);       // the lowest index of the peers is this lane's
        }
    }
}

// ---------------------------------------------------------------------------
// photon-weighted sums of the grouped rays
// ---------------------------------------------------------------------------
// A ray's weight is its content scaled by 2^(28 - e), where 2^e is the power
// of two above its group's largest content (exact power-of-two scaling),
// truncated and at least 1: the brightest member has at least 27 significant
// bits, every weight is below 2^28.  Weighted sums are 64-bit integers.
// Every member of a group of two or more leaves the queue (its slot becomes a
// hole); the leader lists the group in the block's merged-ray list.
__global__ void __launch_bounds__(256, 4) k_mweight(MergeArgs A) {
    __shared__ uint32_t s_wofs[2][9];
    __shared__ int s_on;
    extern __shared__ uint32_t s_drop[];           // per simulation: rays removed
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x) s_drop[k] = 0u;
    Ctl *C = A.ctl;
    if (!block_runs(C, true, &s_on)) return;
    const Queue q = A.q[C->par ^ 1];
    const long long b0 = blockIdx.x * block_chunk(C->cnt[C->par ^ 1]);
    const uint32_t bc = A.w.bcnt[blockIdx.x];
    const int gw = A.w.grp_w;
    const int lane = lane_id();
    uint32_t run = 0;                              // merged rays listed so far (block-uniform)
    for (uint32_t w0 = 0; w0 < bc; w0 += 256) {
        const long long c = b0 + w0 + threadIdx.x;
        const bool in = w0 + threadIdx.x < bc;
        uint4 pk = make_uint4(NO_GROUP, 0u, 0u, 0u);
        uint32_t key = 0, qi = 0;
        if (in) pk = A.w.tgrp[c];
        long long slot = pk.x == NO_GROUP ? -1 : (long long)pk.x;
        uint4 gm = make_uint4(0u, 0u, 0u, 0u);
        if (slot >= 0) gm = A.w.gcm[slot];
        if (slot >= 0 && gm.x < 2u) {
            // alone in its group: the ray stays as it is, and clears the
            // group's word (no other ray touched the group)
            A.w.gcm[slot] = make_uint4(0u, 0u, 0u, 0u);
            slot = -1;
        }
        if (slot >= 0) {
            key = A.w.ckey[c];
            qi = A.w.cand[c];
        }
        const bool leads = slot >= 0 && gm.z == ~(uint32_t)c;
        int sim = -1;
        // a merging member's photons and termination threshold (only rays
        // that merge load them)
        float f[MAXB + 4];
#pragma unroll
        for (int k = 0; k < MAXB + 4; ++k) f[k] = 0.0f;
        int nbf = 0;
        if (slot >= 0) {
            sim = A.nsims > 1 ? A.w.tsim[qi] : 0;
            const SimDev &S = A.sims[sim];
            const uint32_t e = q.em[qi];
            nbf = S.nb;
#pragma unroll
            for (int b = 0; b < MAXB; ++b)
                if (b < nbf) f[b] = q.ph[b][qi];
            const int lev = (int)((pk.y >> 21) & 0xfu);
            const float thr = (e & MERGED_BIT) ? q.mthr[qi]
                                               : S.eps_term * __ldg(&A.em.n0[e]) * pow2_neg(2 * (lev - S.l_src));
#pragma unroll
            for (int b = 0; b <= MAXB; ++b)
                if (b == nbf) f[b] = thr;
            q.pl[qi] = DEAD_RAY;
        }
        unsigned long long v[GSUMS] = {0, 0, 0, 0, 0, 0};
        if (slot >= 0) {
            const int eb = max((int)((gm.y >> 23) & 0xffu), 30);    // biased exponent; 2^(eb-126) > content
            const float wscale = __int_as_float((253 + WBITS - eb) << 23);
            const unsigned long long qw = max(__float2ull_rz(__fmul_rn(__uint_as_float(key), wscale)), 1ull);
            v[0] = qw;
            v[1] = qw * (unsigned long long)(pk.y & 0x1fffffu);
            v[2] = qw * (unsigned long long)(pk.z & 0x1fffffu);
            v[3] = qw * (unsigned long long)(pk.w & 0x1fffffu);
            v[4] = qw * (unsigned long long)((pk.z >> 21) | ((pk.w >> 21) << 11));
            v[5] = qw * (unsigned long long)((pk.y >> 21) & 0xfu);
        }
        const unsigned peers = __match_any_sync(FULL, slot);
        if (__any_sync(FULL, slot >= 0 && __popc(peers) > 1)) {
            peer_sum<GSUMS, unsigned long long>(peers, v);
            peer_sum<MAXB + 4, float>(peers, f);
        }
        if (slot >= 0 && (peers & ((1u << lane) - 1u)) == 0u) {
            unsigned long long *gs = reinterpret_cast<unsigned long long *>(A.w.grp + slot * gw);
#pragma unroll
            for (int k = 0; k < GSUMS; ++k) atomicAdd(gs + k, v[k]);
            float4 *gf = reinterpret_cast<float4 *>(A.w.grp + slot * gw + 2 * GSUMS);
#pragma unroll
            for (int b = 0; b <= MAXB; b += 4)
                if (b <= nbf) red_add_v4(gf + b / 4, f[b], f[b + 1], f[b + 2], f[b + 3]);
        }
        // rays removed: every member of a merging group but one
        const int dsim = slot >= 0 && !leads ? sim : -1;
        if (__any_sync(FULL, dsim >= 0)) {
            const unsigned dp = __match_any_sync(FULL, dsim);
            if (dsim >= 0 && (dp & ((1u << lane) - 1u)) == 0u) atomicAdd(s_drop + dsim, (uint32_t)__popc(dp));
        }
        uint32_t tot;
        const uint32_t r = block_rank(leads, s_wofs[(w0 >> 8) & 1], &tot);
        if (leads) {
            A.w.lead_slot[b0 + run + r] = (uint32_t)slot;
            A.w.lead_sim[b0 + run + r] = sim;
        }
        run += tot;
    }
    if (threadIdx.x == 0) A.w.bled[blockIdx.x] = run;
    __syncthreads();
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x)
        if (s_drop[k]) atomicAdd(A.w.sel + SEL_W * k + SEL_DROP, s_drop[k]);
}

// ---------------------------------------------------------------------------
// the merged rays, appended after the march's output
// ---------------------------------------------------------------------------
// the merged-ray lists' places in the appended run: an exclusive prefix of
// the blocks' counts (written over the candidate counts, which the weight
// pass was the last to read); the queue's new count; the rays the merge
// removed.  One block of 1024 threads, four counts a thread.
__global__ void __launch_bounds__(1024) k_mscan(MergeArgs A, int nblocks) {
    __shared__ unsigned long long s_w[33];
    __shared__ int s_on;
    Ctl *C = A.ctl;
    if (!block_runs(C, true, &s_on)) return;
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    uint32_t v[4];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = 4 * threadIdx.x + j;
        v[j] = k < nblocks ? A.w.bled[k] : 0u;
        sum += v[j];
    }
    const unsigned long long inc = warp_incl_scan64(sum);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const unsigned long long w = s_w[lane], wi = warp_incl_scan64(w);
        __syncwarp();
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    unsigned long long pre = s_w[wid] + inc - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = 4 * threadIdx.x + j;
        if (k < nblocks) A.w.bcnt[k] = (uint32_t)pre;
        pre += v[j];
    }
    const unsigned long long tot = s_w[32];
    const int par = C->par;
    const long long mbase = C->mbase;
    if ((long long)(mbase + tot) > A.cap) {
        if (threadIdx.x == 0) atomicOr(&C->err, 1);
        return;
    }
    if (threadIdx.x == 0) C->cnt[par ^ 1] = mbase + (long long)tot;
    for (int k = threadIdx.x; k < A.nsims; k += blockDim.x) {
        uint32_t *d = A.w.sel + SEL_W * k + SEL_DROP;
        if (*d) {
            A.acc[k].p_rays_out -= (double)*d;
            *d = 0u;
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_memit(MergeArgs A) {
    __shared__ int s_on;
    Ctl *C = A.ctl;
    if (!block_runs(C, true, &s_on)) return;
    const int par = C->par;
    const Queue q = A.q[par ^ 1];
    const long long mbase = C->mbase;
    const unsigned long long pre = A.w.bcnt[blockIdx.x];   // this block's place in the appended run
    const long long b0 = blockIdx.x * block_chunk(mbase);
    const uint32_t bl = A.w.bled[blockIdx.x];
    const int ndir = A.w.ndir, gw = A.w.grp_w, nbq = A.nbq;
    for (uint32_t j = threadIdx.x; j < bl; j += blockDim.x) {
        const uint32_t slot = A.w.lead_slot[b0 + j];
        const int sim = A.w.lead_sim[b0 + j];
        const SimDev &S = A.sims[sim];
        float *gp = A.w.grp + (long long)slot * gw;
        const unsigned long long *gs = reinterpret_cast<const unsigned long long *>(gp);
        const unsigned long long W = gs[0];
        // weights below 2^28 and offsets below 2^21: the sums stay exact
        // while W < 2^41 (more than 2^13 members as bright as the brightest
        // would be needed to reach it)
        if (W >= (1ull << 41)) atomicOr(&C->err, 8);
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
        const long long o = mbase + (long long)pre + j;
        q.pl[o] = ((uint32_t)L2 << LEVEL_SHIFT) | pm;
        q.em[o] = MERGED_BIT | (uint32_t)local;
        q.bi[o] = S.step;
        q.dx[o] = dx; q.dy[o] = dy; q.dz[o] = dz;
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < nbq) q.ph[b][o] = b < S.nb ? gph[b] : 0.0f;
        q.mx[o] = P[0]; q.my[o] = P[1]; q.mz[o] = P[2];
        q.ma[o] = (L2 > S.l_merge ? 0x80000000u : 0u) | ((uint32_t)sim << 16) | (uint32_t)Adist;
        q.mthr[o] = gph[S.nb];
        // the group is cleared for the next step
        float4 *gz = reinterpret_cast<float4 *>(gp);
        for (int b = 0; b < gw / 4; ++b) gz[b] = make_float4(0.f, 0.f, 0.f, 0.f);
        A.w.gcm[slot] = make_uint4(0u, 0u, 0u, 0u);
    }
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

cudaError_t launch_merge(const MergeArgs &a, int sm_count, cudaStream_t st, const MergeSide *side) {
    const int rblocks = std::min(sm_count * 16, MERGE_MAX_BLOCKS);
    const size_t rng_sh = (size_t)(2 * a.nsims + 1) * sizeof(long long) + (size_t)a.nsims * sizeof(int);
    // the merge spheres' rotations depend on no pass of the merge: with a
    // side stream they are drawn (integer-bound) while the selection passes
    // (memory-bound) run, and the group pass waits for both
    cudaError_t e = cudaSuccess;
    if (side) {
        e = cudaEventRecord(side->fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side->st, side->fork, 0);
        if (e != cudaSuccess) return e;
        k_mrot<<<rblocks, 256, rng_sh, side->st>>>(a);
        e = cudaEventRecord(side->join, side->st);
        if (e != cudaSuccess) return e;
    } else {
        k_mrot<<<rblocks, 256, rng_sh, st>>>(a);
    }
    k_mhist1<<<rblocks, 256, 0, st>>>(a);
    if (a.w.hrep > 1) k_mreduce<<<rblocks, 256, 0, st>>>(a, 1);
    k_mfind<<<a.nsims, 1024, 0, st>>>(a, 1);
    k_mhist2<<<rblocks, 256, 0, st>>>(a);
    if (a.w.hrep > 1) k_mreduce<<<rblocks, 256, 0, st>>>(a, 2);
    k_mfind<<<a.nsims, 1024, 0, st>>>(a, 2);
    if (side && (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess) return e;
    k_mgroup<<<rblocks, 256, 0, st>>>(a);
    k_mweight<<<rblocks, 256, (size_t)a.nsims * sizeof(uint32_t), st>>>(a);
    k_mscan<<<1, 1024, 0, st>>>(a, rblocks);
    k_memit<<<rblocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, bool per_ray,
                                     uint32_t *out, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_probe_merge_pixel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(level, n, d, Rq, per_ray ? 1 : 0, out);
    return cudaGetLastError();
}

}  // namespace frt
