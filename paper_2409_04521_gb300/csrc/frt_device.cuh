// frt_device.cuh -- device functions of the RT step.
//
// The HEALPix vectors are computed in double precision with explicitly
// rounded intrinsics (no FMA contraction), so their 2^-24 fixed-point copies
// are the same integers on every IEEE-754 machine that evaluates the same
// expressions in the same order; the sphere rotations are exact integer
// arithmetic.  Everything that decides an integer (directions, crossed
// cells, splits) is integer arithmetic.
#pragma once
#include <cstdint>
#include "frt_types.h"

namespace frt {

constexpr unsigned FULL = 0xffffffffu;
__device__ __constant__ static const double DPI = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// NESTED HEALPix pixel centres (Gorski et al. 2005; Sec. 3.1, Eq. 1)
// ---------------------------------------------------------------------------
// sin x, cos x for x in [0, pi/4]: Taylor series through x^17 / x^18,
// nested so that only exactly rounded + - * / appear.
__device__ __forceinline__ double series_sin(double x) {
    double x2 = __dmul_rn(x, x), t = 1.0;
#pragma unroll
    for (int j = 8; j >= 1; --j) {
        double c = (double)((2 * j) * (2 * j + 1));
        t = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(x2, c), t));
    }
    return __dmul_rn(x, t);
}
__device__ __forceinline__ double series_cos(double x) {
    double x2 = __dmul_rn(x, x), t = 1.0;
#pragma unroll
    for (int j = 9; j >= 1; --j) {
        double c = (double)((2 * j - 1) * (2 * j));
        t = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(x2, c), t));
    }
    return t;
}
// cos(pi m/q), sin(pi m/q) with exact integer reduction to [0, pi/4]
__device__ __forceinline__ void sincos_pi_ratio(long long m, long long q, double &co, double &si) {
    long long M = m % (2 * q);
    if (M < 0) M += 2 * q;
    long long k = (2 * M) / q;
    long long r2 = 4 * M - 2 * k * q;
    double c, s;
    if (r2 <= q) {
        double x = __ddiv_rn(__dmul_rn((double)r2, DPI), (double)(4 * q));
        c = series_cos(x);
        s = series_sin(x);
    } else {
        double x = __ddiv_rn(__dmul_rn((double)(2 * q - r2), DPI), (double)(4 * q));
        c = series_sin(x);
        s = series_cos(x);
    }
    switch ((int)k) {
        case 0: co = c; si = s; break;
        case 1: co = -s; si = c; break;
        case 2: co = -c; si = -s; break;
        default: co = s; si = -c; break;
    }
}

__device__ __forceinline__ long long even_bits(long long v) {
    long long o = 0;
    for (int i = 0; i < 31; ++i)
        if (v & (1LL << (2 * i))) o |= 1LL << i;
    return o;
}

// ring and longitude offsets of the 12 base faces
__device__ __constant__ static const int HP_JR0[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
__device__ __constant__ static const int HP_JP0[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

// unit vector of NESTED pixel p at `level`, as round(v * 2^24)
__device__ inline int4 healpix_vq(int level, long long p) {
    const int *jr0 = HP_JR0, *jp0 = HP_JP0;
    long long ns = 1LL << level, npf = ns * ns;
    long long face = p / npf, ipf = p % npf;
    long long ix = even_bits(ipf), iy = even_bits(ipf >> 1);
    long long jr = jr0[face] * ns - ix - iy - 1;
    long long nr, sh;
    double z;
    if (jr < ns) {
        nr = jr;
        z = __dsub_rn(1.0, __ddiv_rn((double)(nr * nr), (double)(3 * ns * ns)));
        sh = 0;
    } else if (jr > 3 * ns) {
        nr = 4 * ns - jr;
        z = __dsub_rn(__ddiv_rn((double)(nr * nr), (double)(3 * ns * ns)), 1.0);
        sh = 0;
    } else {
        nr = ns;
        z = __ddiv_rn((double)(2 * (2 * ns - jr)), (double)(3 * ns));
        sh = (jr - ns) & 1;
    }
    long long jp = (jp0[face] * nr + ix - iy + 1 + sh) / 2;
    if (jp > 4 * ns) jp -= 4 * ns;
    if (jp < 1) jp += 4 * ns;
    double cp, sp;
    sincos_pi_ratio(2 * jp - sh - 1, 4 * nr, cp, sp);
    double st = __dsqrt_rn(__dmul_rn(__dsub_rn(1.0, z), __dadd_rn(1.0, z)));
    const double Q = 16777216.0;
    return make_int4(__double2int_rn(__dmul_rn(__dmul_rn(st, cp), Q)),
                     __double2int_rn(__dmul_rn(__dmul_rn(st, sp), Q)),
                     __double2int_rn(__dmul_rn(z, Q)), 0);
}

__host__ __device__ __forceinline__ long long level_offset(int l) {  // sum_{j<l} 12*4^j
    return 4LL * ((1LL << (2 * l)) - 1);
}

// ---------------------------------------------------------------------------
// Per-(emitter, step) random rotation (Sec. 3.1), and a cell's merge sphere
// (Sec. 3.3) with the key 2^31 + local cell index.  SplitMix64 (Steele, Lea &
// Flood 2014) as a counter-based stream; each 64-bit draw is read as four
// signed 16-bit integers (w, x, y, z), rejected until 0 < |q|^2 <= 2^30 (a
// uniform integer point of the 4-ball: a uniform unit quaternion by
// direction); the rotation matrix's exact rational entries Q_ij / |q|^2 are
// rounded half to even to 2^-24.  Integer arithmetic only: the same integers
// on every machine, and no double-precision pipe.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
constexpr uint64_t GOLD = 0x9E3779B97F4A7C15ULL;

// num / den rounded half to even, for 0 < den <= 2^30 and |num / den| <= 2^24,
// given rden, the single-precision reciprocal of den: an estimate within a
// few units (three single-precision roundings of a quotient below 2^24)
// corrected exactly by the remainder
__device__ __forceinline__ int32_t div_round_even(long long num, int32_t den, float rden) {
    int32_t q = __float2int_rz((float)num * rden);
    long long r = num - (long long)q * den;
    for (int k = 0; k < 16 && r < 0; ++k) { --q; r += den; }
    for (int k = 0; k < 16 && r >= den; ++k) { ++q; r -= den; }
    if (2 * r > den || (2 * r == den && (q & 1))) ++q;
    return q;
}

__device__ inline void rotation_rows(uint64_t seed, long long e, long long s, int rotate, int4 rows[3]) {
    long long w = 1, x = 0, y = 0, z = 0;
    if (rotate) {
        uint64_t h = sm64(seed + GOLD);
        h = sm64(h + GOLD * (uint64_t)(e + 1));
        h = sm64(h + GOLD * (uint64_t)(s + 1));
        for (int t = 0; t < 64; ++t) {
            const uint64_t u = sm64(h + GOLD * (uint64_t)(t + 1));
            const int a = (int)(u & 0xFFFFu) - 32768, b = (int)((u >> 16) & 0xFFFFu) - 32768;
            const int c = (int)((u >> 32) & 0xFFFFu) - 32768, d = (int)((u >> 48) & 0xFFFFu) - 32768;
            const unsigned n2 = (unsigned)(a * a) + (unsigned)(b * b) + (unsigned)(c * c) + (unsigned)(d * d);
            if (n2 > 0u && n2 <= (1u << 30)) { w = a; x = b; y = c; z = d; break; }
        }
    }
    const long long n = w * w + x * x + y * y + z * z;
    const long long Q[9] = {w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y),
                            2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x),
                            2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z};
    int32_t q[9];
    const float rn = __frcp_rn((float)n);          // one reciprocal for the nine entries
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = div_round_even(Q[i] * (1LL << VQ_BITS), (int32_t)n, rn);
    for (int r = 0; r < 3; ++r) rows[r] = make_int4(q[3 * r], q[3 * r + 1], q[3 * r + 2], 0);
}

// round(X / 2^27), ties to even (X = Rq . vq, 2^48 scale -> 2^21 scale)
__device__ __forceinline__ int32_t rne_shift27(long long X) {
    long long q = X >> 27;                 // arithmetic shift = floor
    long long r = X - (q << 27);
    const long long half = 1LL << 26;
    q += (r > half) | ((r == half) & (q & 1));
    return (int32_t)q;
}
__device__ __forceinline__ void rotate_dir(const int4 rows[3], int4 v, int32_t &dx, int32_t &dy, int32_t &dz) {
    dx = rne_shift27((long long)rows[0].x * v.x + (long long)rows[0].y * v.y + (long long)rows[0].z * v.z);
    dy = rne_shift27((long long)rows[1].x * v.x + (long long)rows[1].y * v.y + (long long)rows[1].z * v.z);
    dz = rne_shift27((long long)rows[2].x * v.x + (long long)rows[2].y * v.y + (long long)rows[2].z * v.z);
}

// ---------------------------------------------------------------------------
// Merge-sphere pixel (Sec. 3.3).  The pixel decides which rays merge, so it
// is computed in single precision as one fixed sequence of correctly rounded
// operations (explicit _rn intrinsics: nothing is contracted into an FMA):
// v = Rq^T d, then the NESTED HEALPix ang2pix (Gorski et al. 2005) with the
// azimuth from an arctangent series.  The quantised rotation entries
// (|Rq| <= 2^24) and the fixed-point direction (|d| <= 2^21) are exact floats.
// ---------------------------------------------------------------------------
// arctan(t) / (pi/2), 0 <= t <= 1: t > tan(pi/8) uses arctan t = pi/4 +
// arctan((t-1)/(t+1)); then Taylor terms u^(2k+1)/(2k+1), k = 0..9.
__device__ __forceinline__ float atan_quarter(float t) {
    const float c[10] = {1.0f, -0.333333343f, 0.200000003f, -0.142857149f, 0.111111112f,
                         -0.0909090936f, 0.0769230798f, -0.0666666701f, 0.0588235296f, -0.0526315793f};
    float base = 0.0f, u = t;
    if (t > 0.414213568f) {
        u = __fdiv_rn(__fadd_rn(t, -1.0f), __fadd_rn(t, 1.0f));
        base = 0.5f;
    }
    const float u2 = __fmul_rn(u, u);
    float p = c[9];
#pragma unroll
    for (int k = 8; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, u2), c[k]);
    return __fadd_rn(base, __fmul_rn(__fmul_rn(u, p), 0.636619747f));
}
// azimuth of (x, y) in quarter turns, [0, 4)
__device__ __forceinline__ float azimuth_quarter(float x, float y) {
    const float ax = fabsf(x), ay = fabsf(y);
    if (ax == 0.0f && ay == 0.0f) return 0.0f;
    const float a = ax >= ay ? atan_quarter(__fdiv_rn(ay, ax)) : __fadd_rn(1.0f, -atan_quarter(__fdiv_rn(ax, ay)));
    float tt;
    if (x >= 0.0f) tt = y >= 0.0f ? a : __fadd_rn(4.0f, -a);
    else tt = y >= 0.0f ? __fadd_rn(2.0f, -a) : __fadd_rn(2.0f, a);
    if (tt >= 4.0f) tt = __fadd_rn(tt, -4.0f);
    return tt;
}
__device__ __forceinline__ uint32_t interleave_bits(uint32_t ix, uint32_t iy) {
    uint32_t out = 0;
    for (int i = 0; i < 13; ++i) out |= (((ix >> i) & 1u) << (2 * i)) | (((iy >> i) & 1u) << (2 * i + 1));
    return out;
}
// NESTED pixel at `level` (<= 12) of fixed-point direction d on the sphere
// whose pixel vectors are rotated by `rows` (d = Rq . v, so v = Rq^T d)
__device__ __forceinline__ uint32_t merge_pixel(int level, const int4 rows[3], int32_t dx, int32_t dy, int32_t dz) {
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float v0 = __fadd_rn(__fadd_rn(__fmul_rn((float)rows[0].x, fx), __fmul_rn((float)rows[1].x, fy)),
                               __fmul_rn((float)rows[2].x, fz));
    const float v1 = __fadd_rn(__fadd_rn(__fmul_rn((float)rows[0].y, fx), __fmul_rn((float)rows[1].y, fy)),
                               __fmul_rn((float)rows[2].y, fz));
    const float v2 = __fadd_rn(__fadd_rn(__fmul_rn((float)rows[0].z, fx), __fmul_rn((float)rows[1].z, fy)),
                               __fmul_rn((float)rows[2].z, fz));
    const int nside = 1 << level;
    const float ns = (float)nside;
    const float s2 = __fadd_rn(__fmul_rn(v0, v0), __fmul_rn(v1, v1));
    const float r = __fsqrt_rn(__fadd_rn(s2, __fmul_rn(v2, v2)));
    const float z = __fdiv_rn(v2, r);
    const float tt = azimuth_quarter(v0, v1);
    int face, ix, iy;
    if (fabsf(z) <= 0.666666687f) {                  // equatorial belt
        const float t1 = __fmul_rn(ns, __fadd_rn(0.5f, tt));
        const float t2 = __fmul_rn(ns, __fmul_rn(z, 0.75f));
        const int jp = (int)__fadd_rn(t1, -t2), jm = (int)__fadd_rn(t1, t2);
        const int ifp = jp >> level, ifm = jm >> level;
        face = ifp == ifm ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
        ix = jm & (nside - 1);
        iy = nside - (jp & (nside - 1)) - 1;
    } else {                                         // polar caps
        int ntt = (int)tt;
        if (ntt > 3) ntt = 3;
        const float tp = __fadd_rn(tt, -(float)ntt);
        const float omz = __fdiv_rn(s2, __fmul_rn(r, __fadd_rn(r, fabsf(v2))));   // 1 - |z|
        const float tmp = __fmul_rn(ns, __fsqrt_rn(__fmul_rn(3.0f, omz)));
        int jp = (int)__fmul_rn(tp, tmp), jm = (int)__fmul_rn(__fadd_rn(1.0f, -tp), tmp);
        jp = min(jp, nside - 1);
        jm = min(jm, nside - 1);
        if (z >= 0.0f) { face = ntt; ix = nside - jm - 1; iy = nside - jp - 1; }
        else { face = ntt + 8; ix = jp; iy = jm; }
    }
    return (uint32_t)face * (uint32_t)(nside * nside) + interleave_bits((uint32_t)ix, (uint32_t)iy);
}

// Split children of a merged ray of level l centred on merge pixel pm (level
// lm <= l).  A NESTED pixel's centre is the corner its four children share,
// and at each deeper level the corner of exactly four pixels: child i, then
// always sub-pixel 3-i.  Child c of an m-level split is descendant
// c mod 4^(m-1) of the (c >> 2(m-1))-th of these level-(l+1) pixels.
__device__ __forceinline__ uint32_t vertex_child(int lm, uint32_t pm, int l, int m, uint32_t c) {
    const uint32_t i = c >> (2 * (m - 1)), j = c & ((1u << (2 * (m - 1))) - 1u);
    uint32_t q = pm * 4u + i;
    for (int k = l - lm; k > 0; --k) q = q * 4u + (3u - i);
    return (q << (2 * (m - 1))) + j;
}

// ---------------------------------------------------------------------------
// One-step traversal (Sec. 3.1): the segment p0 -> p0 + d through unit cells.
// Integer state; a ray on a face belongs to the cell it moves into; tied face
// crossings step together; the order of the crossings is decided by exact
// integer comparisons.
// ---------------------------------------------------------------------------
// exact 32x32 -> 64-bit unsigned product (one wide multiply)
__device__ __forceinline__ unsigned long long wmul(unsigned a, unsigned b) { return (unsigned long long)a * b; }

// exact single-precision value of an unsigned integer below 2^23, on the
// integer and FMA pipes (no conversion instruction)
__device__ __forceinline__ float u23_to_float(unsigned u) {
    return __fadd_rn(__uint_as_float(0x4B000000u | u), -8388608.0f);
}

struct Walk {
    int cx, cy, cz;          // current cell
    unsigned Dx, Dy, Dz;     // distance along each axis to the next face ahead (<= 2^21)
    unsigned ax, ay, az;     // |d| (<= 2^21)
    int sx, sy, sz;          // sign of d
};

// cell index (floor) and distance to the next face for one axis; a ray on a
// face belongs to the cell it moves into
__device__ __forceinline__ void axis_init(int p, int d, int &c, unsigned &D, unsigned &a, int &s) {
    const unsigned MASK = (unsigned)ONE_CELL - 1u;
    if (d > 0) {
        c = p >> FRAC_BITS; D = (unsigned)ONE_CELL - ((unsigned)p & MASK); a = (unsigned)d; s = 1;
    } else if (d < 0) {
        const int q = p - 1;
        c = q >> FRAC_BITS; D = ((unsigned)q & MASK) + 1u; a = (unsigned)(-d); s = -1;
    } else {
        c = p >> FRAC_BITS; D = 0u; a = 0u; s = 0;
    }
}
// positions in 2^-21 cell, |p| < 2^31 - 2^21 (a ray within 1000 cells of the
// box; arithmetic right shifts are floors)
__device__ __forceinline__ void walk_init(Walk &w, int px, int py, int pz, int dx, int dy, int dz) {
    axis_init(px, dx, w.cx, w.Dx, w.ax, w.sx);
    axis_init(py, dy, w.cy, w.Dy, w.ay, w.sy);
    axis_init(pz, dz, w.cz, w.Dz, w.az, w.sz);
}
__device__ __forceinline__ bool walk_outside(const Walk &w, int nx, int ny, int nz) {
    return (unsigned)w.cx >= (unsigned)nx || (unsigned)w.cy >= (unsigned)ny || (unsigned)w.cz >= (unsigned)nz;
}
// The segments of one step.  |d_a| is at most one cell, so each axis is
// crossed at most once, at t_a = D_a/|d_a| < 1 (D_a < |d_a|); the segments
// end at these times in increasing order and at t = 1.  The order is decided
// once per step by exact cross-multiplied comparisons (the rank of an axis:
// the crossing axes strictly earlier); axes crossed at the same t step
// together.  A segment from t_p = D_p/a_p to t_c = D_c/a_c has the length
// (D_c a_p - D_p a_c) / (a_c a_p): the numerator, an integer below 2^44, is
// formed in single precision with the exact rounding errors of its two
// products (fma), so it is within an ulp; times the approximate
// reciprocals of a_c and a_p the length is within a few ulp of the exact
// fraction, however short it is (D, a <= 2^21 are exact floats, converted
// on the integer and FMA pipes).  Outputs by fixed slot, so that they stay
// in registers: slot r < 3 holds the segment that ends at the crossing of
// rank r, slot 3 the one that ends the step; the bits of the returned mask
// mark the slots in use (none after the ray leaves the grid: esc), in order
// along the ray.  A slot's cell is key = coff + (z ny + y) nx + x (-1 for an
// empty slot).
__device__ __forceinline__ float cross_diff(float dc, float ap, float dp, float ac) {
    const float p1 = __fmul_rn(dc, ap), p2 = __fmul_rn(dp, ac);
    const float e1 = __fmaf_rn(dc, ap, -p1), e2 = __fmaf_rn(dp, ac, -p2);
    return __fadd_rn(__fadd_rn(p1, -p2), __fadd_rn(e1, -e2));
}
__device__ __forceinline__ unsigned walk_step(const Walk &w, int nx, int ny, int nz, int coff, int (&key)[4],
                                              float (&ds)[4], bool &esc) {
#pragma unroll
    for (int r = 0; r < 4; ++r) { key[r] = -1; ds[r] = 0.0f; }
    esc = walk_outside(w, nx, ny, nz);
    if (esc) return 0u;
    const bool crx = w.sx != 0 && w.Dx < w.ax;
    const bool cry = w.sy != 0 && w.Dy < w.ay;
    const bool crz = w.sz != 0 && w.Dz < w.az;
    // t_i < t_j  <=>  D_i |d_j| < D_j |d_i|
    const unsigned long long xy = wmul(w.Dx, w.ay), yx = wmul(w.Dy, w.ax);
    const unsigned long long xz = wmul(w.Dx, w.az), zx = wmul(w.Dz, w.ax);
    const unsigned long long yz = wmul(w.Dy, w.az), zy = wmul(w.Dz, w.ay);
    const int rx = (cry && yx < xy) + (crz && zx < xz);
    const int ry = (crx && xy < yx) + (crz && zy < yz);
    const int rz = (crx && xz < zx) + (cry && yz < zy);
    // the crossing axes' D, |d| and 1/|d| in single precision
    const float fDx = u23_to_float(w.Dx), fDy = u23_to_float(w.Dy), fDz = u23_to_float(w.Dz);
    const float fax = u23_to_float(w.ax), fay = u23_to_float(w.ay), faz = u23_to_float(w.az);
    const float rax = crx ? __fdividef(1.0f, fax) : 0.0f;
    const float ray = cry ? __fdividef(1.0f, fay) : 0.0f;
    const float raz = crz ? __fdividef(1.0f, faz) : 0.0f;
    int x = w.cx, y = w.cy, z = w.cz;
    float dp = 0.0f, ap = 1.0f, rp = 1.0f;     // end of the previous segment: t = dp / ap
    unsigned mask = 0u;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const bool bx = crx && rx == r, by = cry && ry == r, bz = crz && rz == r;
        key[r] = -1;
        ds[r] = 0.0f;
        if (!esc && (bx || by || bz)) {
            key[r] = coff + (z * ny + y) * nx + x;
            const float dc = bx ? fDx : (by ? fDy : fDz);
            const float ac = bx ? fax : (by ? fay : faz);
            const float rc = bx ? rax : (by ? ray : raz);
            ds[r] = __fmul_rn(__fmul_rn(cross_diff(dc, ap, dp, ac), rc), rp);
            mask |= 1u << r;
            if (bx) x += w.sx;
            if (by) y += w.sy;
            if (bz) z += w.sz;
            dp = dc; ap = ac; rp = rc;
            esc = (unsigned)x >= (unsigned)nx || (unsigned)y >= (unsigned)ny || (unsigned)z >= (unsigned)nz;
        }
    }
    key[3] = -1;
    ds[3] = 0.0f;
    if (!esc) {
        key[3] = coff + (z * ny + y) * nx + x;
        ds[3] = __fmul_rn(__fadd_rn(ap, -dp), rp);      // (a_p - D_p) / a_p, exact numerator
        mask |= 8u;
    }
    return mask;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Sum NV values over the lanes of each peer group (lanes with the same key);
// the lowest lane of each group ends with the group sum.  Pairwise tree over
// the ranks within each group: log2(group size) rounds.
template <int NV, typename T = float>
__device__ __forceinline__ void peer_sum(unsigned peers, T (&v)[NV]) {
    const int lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    unsigned above = lane == 31 ? 0u : (peers & (0xffffffffu << (lane + 1)));
    int rank = __popc(peers & below);
    bool alive = true;
    while (__any_sync(FULL, alive && above != 0u)) {
        int src = above ? (__ffs(above) - 1) : lane;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T t = __shfl_sync(FULL, v[k], src);
            if (alive && !(rank & 1) && above) v[k] += t;
        }
        unsigned odd = __ballot_sync(FULL, alive && (rank & 1));
        if (rank & 1) alive = false;
        above &= ~odd;
        rank >>= 1;
    }
}

// Sum NV values over runs of equal consecutive keys (segmented shuffle
// tree); the first lane of each run ends with the run's sum.  Equal keys that
// are not adjacent stay in separate runs.
template <int NV>
__device__ __forceinline__ bool run_sum(int key, float (&v)[NV]) {
    const int lane = lane_id();
    const int prev = __shfl_up_sync(FULL, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const unsigned above = lane == 31 ? 0u : (heads & (0xffffffffu << (lane + 1)));
    const int run_end = above ? __ffs(above) - 1 : 32;
    if (__all_sync(FULL, run_end == lane + 1)) return head;   // all runs of length 1
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float t = __shfl_down_sync(FULL, v[k], d);
            if (lane + d < run_end) v[k] += t;
        }
    }
    return head;
}

// Sum NV values over the whole warp (butterfly); every lane gets the sum.
template <int NV, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[NV]) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(FULL, v[k], d);
    }
}

// Warp-inclusive prefix sum of an int.
__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    return x;
}

// exact 2^-k for 0 <= k < 126
__device__ __forceinline__ float pow2_neg(int k) { return __int_as_float((127 - k) << 23); }

// v * 2^32 rounded to an unsigned 64-bit integer, for v >= 0 below 2^31;
// built from the float's bits (no 64-bit conversion instruction)
__device__ __forceinline__ unsigned long long fixed32(float v) {
    const unsigned b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0 || (b >> 31)) return 0ull;
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 118;                      // value * 2^32 = m * 2^(e - 150 + 32)
    if (sh >= 0) return sh < 40 ? (m << sh) : 0xffffffffffffffffull;
    const int r = -sh;
    if (r > 24) return 0ull;
    return (m + (1ull << (r - 1))) >> r;
}

__device__ __forceinline__ void red_add_v2(float2 *addr, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Rate coefficients in single precision (temperature-dependent fits cited by
// Sec. 4.1: Hui & Gnedin 1997 for case-B recombination, recombination cooling
// and collisional ionisation; Cen 1992 for collisional excitation and
// free-free cooling; Compton cooling from physical constants).
// ---------------------------------------------------------------------------
constexpr float KB_F = 1.380649e-16f;
constexpr float T_HI_F = 157807.0f;

// The fits are evaluated in log2 space: with t = log2 T and l = log2 lambda
// (lambda = 2 T_HI / T), every power, quotient and Boltzmann factor is one
// exp2 of a sum, and T's logarithm is taken once.  Hardware log2/exp2: the
// exponents stay below ~30 in magnitude (the large constant factors are kept
// outside), so each rate is within a few 1e-6 relative of the fit.
constexpr float LOG2_2THI = 18.2678017f;           // log2(2 T_HI)
constexpr float HALF_LOG2E = 0.721347520f;         // log2(e) / 2

// log2 of (1 + (lambda / b)^c)^d from l = log2 lambda and lb = log2 b
__device__ __forceinline__ float hg_den(float l, float lb, float c, float d) {
    return d * __log2f(1.0f + exp2f(c * (l - lb)));
}
__device__ __forceinline__ float alphaB_f(float T) {
    const float l = LOG2_2THI - __log2f(T);
    return 2.753e-14f * exp2f(1.5f * l - hg_den(l, 1.45417589f, 0.407f, 2.242f));      // b = 2.740
}
// case-A recombination coefficient (Hui & Gnedin 1997)
__device__ __forceinline__ float alphaA_f(float T) {
    const float l = LOG2_2THI - __log2f(T);
    return 1.269e-13f * exp2f(1.503f * l - hg_den(l, -0.937878288f, 0.470f, 1.923f));  // b = 0.522
}
// collisional ionisation rate from t = log2 T, l = log2 lambda and lambda
__device__ __forceinline__ float collion_tl(float t, float l, float lam) {
    if (lam > 180.0f) return 0.0f;                    // exp(-lam/2) below the float range
    return 21.11f * exp2f(-1.5f * t - HALF_LOG2E * lam - 1.089f * l - hg_den(l, -1.49817873f, 0.874f, 1.101f));
}
__device__ __forceinline__ float collion_f(float T) {
    const float t = __log2f(T), l = LOG2_2THI - t;
    return collion_tl(t, l, exp2f(l));
}
// net cooling rate per n_H^2 (erg cm^3 s^-1) for electron, HI and HII
// fractions xe, xHI, xHII; compton_c already divided by n_H
__device__ __forceinline__ float cooling_f(float T, float xe, float xHI, float xHII, float compton_c, float Tcmb) {
    const float t = __log2f(T), l = LOG2_2THI - t, lam = exp2f(l);
    // recombination cooling: T lambda^1.970 / (1 + (lambda/2.250)^0.376)^3.720
    const float rec = 3.435e-30f * exp2f(t + 1.970f * l - hg_den(l, 1.169925f, 0.376f, 3.720f));
    const float cion = 2.1789874e-11f * collion_tl(t, l, lam);     // 13.6 eV in erg
    // collisional excitation: exp(-118348 / T) / (1 + sqrt(T / 1e5)), and
    // 118348 / T = 0.374976 lambda
    const float cexc = 7.5e-19f * exp2f(-0.540977500f * lam - __log2f(1.0f + exp2f(0.5f * (t - 16.6096405f))));
    const float u = 5.5f - 0.301029996f * t;                         // 5.5 - log10 T
    const float gff = 1.1f + 0.34f * exp2f(-0.480898347f * u * u);  // exp(-u^2 / 3)
    const float ff = 1.42e-27f * gff * exp2f(0.5f * t);
    return (rec + ff) * xe * xHII + (cion + cexc) * xe * xHI + compton_c * (T - Tcmb) * xe;
}

}  // namespace frt
