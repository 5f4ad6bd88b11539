/*
 * flexrt_oracle.c -- plain, slow, FP64 CPU oracle of the FlexRT adaptive
 * ray-tracing radiative-transfer step (Cain & D'Aloisio, arXiv:2409.04521).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path; the two
 * agree only because both follow the same reading of the paper.
 *
 * Everything here is double precision in physical cgs units, written in the
 * order the paper states the method:
 *   Sec. 3.1, Eq. 1  -- 12*4^l HEALPix rays cast from the centre of every
 *                       source cell, NESTED pixel numbering, a fresh random
 *                       rotation of each source's sphere every step;
 *   Sec. 3.1         -- each ray moves exactly one cell width per step and is
 *                       absorbed in every cell it crosses;
 *   Sec. 3.2, Eq. 2-3 -- a level-l ray splits into (l+1, 4p+i), i=0..3, once
 *                       its distance from the source reaches r_split(l);
 *   Sec. 3.3, Eq. 4  -- optional ray merging at the end of each step: the
 *                       N_ex*N_RT brightest rays are exempt, the others merge
 *                       per (cell, pixel of a randomly oriented level-l_merge
 *                       sphere of that cell);
 *   Sec. 4.2, Eq. 13 and 17 -- tau = kappa*ds and the cell-averaged
 *                       photo-ionisation rate for a finite mean free path
 *                       (kappa = n_HI sigma + 1/lambda_mfp);
 *   Sec. 4.1, Eq. 6-11 -- C2-Ray style time-dependent ionisation update,
 *                       optionally iterated with the march (Gamma from the
 *                       time-averaged n_HI, Eq. 11);
 *   Sec. 4.1, Eq. 12 -- temperature equation (static density, fixed z);
 *   Sec. 4.2, Eq. 14-19 -- optional Generalized Opacity mode: a cell is a
 *                       highly ionised fraction x_ion with the sub-grid
 *                       opacity and a neutral rest behind an infinitely thin
 *                       moving screen that the photons reaching it advance.
 *   Sec. 4.2, Eq. 20-22 -- in that mode the photo-ionisation-equilibrium
 *                       opacity law and, with evolving temperature, newly
 *                       ionised gas at T_reion heated by the power-law
 *                       photo-heating of Eq. 22 (helium singly ionised with
 *                       hydrogen through chi, Eq. 18).
 * Where the paper is silent the reading taken is stated at the spot
 * (fixed-point geometry, termination, rotation sampler, rate fits ...).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction:
 * the HEALPix vectors and rotations must be the correctly rounded result of
 * every written operation, in the written order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_FRAC_BITS 21                     /* positions: 2^-21 cell units      */
#define OR_S ((int64_t)1 << OR_FRAC_BITS)   /* one cell in fixed point          */
#define OR_VQ_BITS 24                       /* pixel vectors / rotation entries */
#define OR_MAXB 8                           /* max frequency bins               */
#define OR_MAXL 13                          /* levels 0..12                     */

static const double OR_PI = 3.141592653589793238462643383279502884;

/* ------------------------------------------------------------------------- */
/* integer helpers                                                            */
/* ------------------------------------------------------------------------- */
static int64_t floordiv64(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* round(X / 2^k) with ties to even, exact integer arithmetic */
static int64_t rne_shift(int64_t X, int k)
{
    int64_t den = (int64_t)1 << k;
    int64_t q = floordiv64(X, den);
    int64_t r = X - q * den;           /* 0 <= r < den */
    int64_t half = den >> 1;
    if (r > half) q += 1;
    else if (r == half && (q & 1)) q += 1;
    return q;
}

/* ------------------------------------------------------------------------- */
/* HEALPix NESTED pix2vec (Gorski et al. 2005, cited in Sec. 3.1)             */
/* ------------------------------------------------------------------------- */

/* sin and cos on [0, pi/4] by their Taylor series (through x^17 and x^18),
 * nested so that only + - * / by exact integers appear. */
static double taylor_sin(double x)
{
    double x2 = x * x, t = 1.0;
    for (int j = 8; j >= 1; --j) {
        double c = (double)((2 * j) * (2 * j + 1));
        double a = x2 / c;
        double b = a * t;
        t = 1.0 - b;
    }
    return x * t;
}
static double taylor_cos(double x)
{
    double x2 = x * x, t = 1.0;
    for (int j = 9; j >= 1; --j) {
        double c = (double)((2 * j - 1) * (2 * j));
        double a = x2 / c;
        double b = a * t;
        t = 1.0 - b;
    }
    return t;
}

/* cos(pi m / q), sin(pi m / q) for integers m, q > 0: exact integer quadrant
 * reduction, then the series on an argument in [0, pi/4]. */
static void sincos_pi_frac(int64_t m, int64_t q, double *co, double *si)
{
    int64_t M = m % (2 * q);
    if (M < 0) M += 2 * q;                 /* angle pi*M/q in [0, 2pi)        */
    int64_t k = (2 * M) / q;               /* quadrant 0..3                   */
    int64_t r2 = 4 * M - 2 * k * q;        /* psi = pi*r2/(4q) in [0, pi/2)   */
    double c, s;
    if (r2 <= q) {
        double x = ((double)r2 * OR_PI) / (double)(4 * q);
        c = taylor_cos(x);
        s = taylor_sin(x);
    } else {
        double x = ((double)(2 * q - r2) * OR_PI) / (double)(4 * q);
        c = taylor_sin(x);
        s = taylor_cos(x);
    }
    switch ((int)k) {
    case 0: *co = c;  *si = s;  break;
    case 1: *co = -s; *si = c;  break;
    case 2: *co = -c; *si = -s; break;
    default: *co = s; *si = -c; break;
    }
}

static const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

static int64_t compact_even_bits(int64_t v)
{
    int64_t out = 0;
    for (int i = 0; i < 31; ++i)
        if (v & ((int64_t)1 << (2 * i))) out |= (int64_t)1 << i;
    return out;
}

/* unit vector of NESTED pixel p at level l (nside = 2^l) */
int or_pix2vec(int level, int64_t p, double v[3])
{
    if (level < 0 || level >= OR_MAXL) return -1;
    int64_t nside = (int64_t)1 << level, npface = nside * nside;
    if (p < 0 || p >= 12 * npface) return -1;
    int64_t face = p / npface, ipf = p % npface;
    int64_t ix = compact_even_bits(ipf), iy = compact_even_bits(ipf >> 1);
    int64_t jr = jrll[face] * nside - ix - iy - 1;
    int64_t nr, kshift;
    double z;
    if (jr < nside) {
        nr = jr;
        z = 1.0 - (double)(nr * nr) / (double)(3 * nside * nside);
        kshift = 0;
    } else if (jr > 3 * nside) {
        nr = 4 * nside - jr;
        z = (double)(nr * nr) / (double)(3 * nside * nside) - 1.0;
        kshift = 0;
    } else {
        nr = nside;
        z = (double)(2 * (2 * nside - jr)) / (double)(3 * nside);
        kshift = (jr - nside) & 1;
    }
    int64_t jp = (jpll[face] * nr + ix - iy + 1 + kshift) / 2;
    if (jp > 4 * nside) jp -= 4 * nside;
    if (jp < 1) jp += 4 * nside;
    /* phi = (jp - (kshift+1)/2) * pi / (2 nr) = pi * (2 jp - kshift - 1) / (4 nr) */
    double cp, sp;
    sincos_pi_frac(2 * jp - kshift - 1, 4 * nr, &cp, &sp);
    double st = sqrt((1.0 - z) * (1.0 + z));
    v[0] = st * cp;
    v[1] = st * sp;
    v[2] = z;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Random rotation of a source's HEALPix sphere (Sec. 3.1).                   */
/* Reading: one uniform rotation per (seed, emitter, step).  The draws come   */
/* from SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based stream; */
/* each 64-bit draw is read as four signed 16-bit integers (w, x, y, z), and  */
/* draws are rejected until 0 < w^2+x^2+y^2+z^2 <= 2^30: a uniform integer    */
/* point of the 4-ball, whose direction is a uniform unit quaternion (the     */
/* rejection idea of Marsaglia 1972, in integers).  The rotation matrix of    */
/* that quaternion has the exact rational entries Q_ij / n, n = |q|^2, which  */
/* are rounded half to even to 2^-24 in exact integer arithmetic: no step     */
/* rounds anything but that last one, so the sphere is the same on every      */
/* machine.                                                                   */
/* ------------------------------------------------------------------------- */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;
static uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static uint64_t rot_key(uint64_t seed, int64_t e, int64_t s)
{
    uint64_t h = sm_mix(seed + SM_GAMMA);
    h = sm_mix(h + SM_GAMMA * (uint64_t)(e + 1));
    h = sm_mix(h + SM_GAMMA * (uint64_t)(s + 1));
    return h;
}

/* raw 64-bit draw i of the stream keyed by `key` (exposed for tests) */
uint64_t or_sm_draw(uint64_t key, int32_t i) { return sm_mix(key + SM_GAMMA * (uint64_t)(i + 1)); }
uint64_t or_rot_key(uint64_t seed, int64_t e, int64_t s) { return rot_key(seed, e, s); }

/* num / den rounded to nearest, ties to even, for den > 0 */
static int64_t div_round_even(int64_t num, int64_t den)
{
    int64_t q = num / den, r = num % den;          /* C: truncation toward zero */
    if (r < 0) { q -= 1; r += den; }               /* floor and 0 <= r < den     */
    if (2 * r > den || (2 * r == den && (q & 1))) q += 1;
    return q;
}

/* rotation matrix R (row major, Q_ij / n) and its 2^24 fixed-point copy */
void or_rotation(uint64_t seed, int64_t e, int64_t s, int rotate, double R[9], int32_t Rq[9])
{
    int64_t w = 1, x = 0, y = 0, z = 0;
    if (rotate) {
        const uint64_t key = rot_key(seed, e, s);
        for (int t = 0; t < 64; ++t) {
            const uint64_t u = or_sm_draw(key, t);
            const int64_t a = (int64_t)((u >> 0) & 0xFFFF) - 32768, b = (int64_t)((u >> 16) & 0xFFFF) - 32768;
            const int64_t c = (int64_t)((u >> 32) & 0xFFFF) - 32768, d = (int64_t)((u >> 48) & 0xFFFF) - 32768;
            const int64_t n2 = a * a + b * b + c * c + d * d;
            if (n2 > 0 && n2 <= ((int64_t)1 << 30)) { w = a; x = b; y = c; z = d; break; }
        }
    }
    const int64_t n = w * w + x * x + y * y + z * z;
    const int64_t Q[9] = {w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y),
                          2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x),
                          2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z};
    for (int i = 0; i < 9; ++i) {
        R[i] = (double)Q[i] / (double)n;
        Rq[i] = (int32_t)div_round_even(Q[i] * ((int64_t)1 << OR_VQ_BITS), n);
    }
}

/* Random rotation of a cell's merge sphere (Sec. 3.3: "in each cell, we
 * throw down a randomly oriented HealPix sphere").  Drawn exactly like an
 * emitter's sphere (or_rotation: the same counter-based stream and Marsaglia
 * quaternion in double precision) with the key 2^31 + local cell index, one
 * per (cell, step).  Rq = round(R * 2^24). */
#define OR_MERGE_KEY ((int64_t)1 << 31)
void or_merge_rotation(uint64_t seed, int64_t cell, int64_t s, int rotate, int32_t Rq[9])
{
    double R[9];
    or_rotation(seed, OR_MERGE_KEY + cell, s, rotate, R, Rq);
}

int or_direction(int level, int64_t p, const int32_t Rq[9], int32_t d[3])
{
    double v[3];
    if (or_pix2vec(level, p, v)) return -1;
    int64_t vq[3];
    for (int j = 0; j < 3; ++j) vq[j] = (int64_t)nearbyint(v[j] * 16777216.0);
    for (int a = 0; a < 3; ++a) {
        int64_t acc = 0;
        for (int j = 0; j < 3; ++j) acc += (int64_t)Rq[3 * a + j] * vq[j];
        d[a] = (int32_t)rne_shift(acc, 2 * OR_VQ_BITS - OR_FRAC_BITS);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Split radius table (Sec. 3.2, Eq. 2) in whole steps:                       */
/* K[l] = smallest integer k >= 1 with k >= 2^l sqrt(3/(pi N_min)).           */
/* The ray has travelled (age+1) cells after its march; it splits while       */
/* age+1 >= K[l].                                                             */
/* ------------------------------------------------------------------------- */
void or_split_table(double n_min, int32_t K[OR_MAXL])
{
    double f = sqrt(3.0 / (OR_PI * n_min));
    for (int l = 0; l < OR_MAXL; ++l) {
        double r = ldexp(f, l);
        int64_t k = (int64_t)ceil(r);
        if (k < 1) k = 1;
        K[l] = (int32_t)k;
    }
}

/* ------------------------------------------------------------------------- */
/* Cell traversal of one step (Sec. 3.1): the segment from p0 to p0 + d.      */
/* Reading: the crossed cells are those of the exact straight segment; a ray  */
/* sitting on a face belongs to the cell it moves into; simultaneous face     */
/* crossings step all those axes at once (no zero-length segment); the step   */
/* ends at t = 1 and a face reached exactly at t = 1 is crossed next step.    */
/* t runs over [0,1] and one step is one cell width, so ds = dt in cells.     */
/* Returns the number of in-box segments; *escaped = 1 if the ray left the    */
/* box [0,n)^3 (open boundaries).                                             */
/* ------------------------------------------------------------------------- */
/* Merge-sphere pixel of a direction (Sec. 3.3)                               */
/* ------------------------------------------------------------------------- */
/* The pixel a ray "occupies" on the randomly oriented level-l_merge sphere
 * of its cell: the NESTED ang2pix of Gorski et al. (2005) of the direction
 * expressed in the sphere's own frame, v = Rq^T d (the sphere's pixel
 * vectors are Rq . v), in double precision with the library atan2. */

static int64_t spread_bits(int64_t v) /* bit i of v to bit 2i */
{
    int64_t out = 0;
    for (int i = 0; i < 31; ++i)
        if (v & ((int64_t)1 << i)) out |= (int64_t)1 << (2 * i);
    return out;
}

int64_t or_merge_pixel(int level, const int32_t Rq[9], const int32_t d[3])
{
    double v[3];
    for (int j = 0; j < 3; ++j)    /* integers below 2^47: exact */
        v[j] = (double)Rq[j] * (double)d[0] + (double)Rq[3 + j] * (double)d[1] + (double)Rq[6 + j] * (double)d[2];
    const int64_t nside = (int64_t)1 << level;
    const double ns = (double)nside;
    const double s2 = v[0] * v[0] + v[1] * v[1];
    const double r = sqrt(s2 + v[2] * v[2]);
    const double z = v[2] / r, za = fabs(z);
    double tt = atan2(v[1], v[0]) / (0.5 * OR_PI);   /* azimuth in quarter turns */
    if (tt < 0.0) tt += 4.0;
    if (tt >= 4.0) tt -= 4.0;
    int64_t face, ix, iy;
    if (za <= 2.0 / 3.0) {                          /* equatorial belt */
        const double t1 = ns * (0.5 + tt), t2 = ns * z * 0.75;
        const int64_t jp = (int64_t)(t1 - t2), jm = (int64_t)(t1 + t2);
        const int64_t ifp = jp >> level, ifm = jm >> level;
        face = ifp == ifm ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
        ix = jm & (nside - 1);
        iy = nside - (jp & (nside - 1)) - 1;
    } else {                                         /* polar caps */
        int64_t ntt = (int64_t)tt;
        if (ntt > 3) ntt = 3;
        const double tp = tt - (double)ntt;
        const double omz = s2 / (r * (r + fabs(v[2])));   /* 1 - |z| */
        const double tmp = ns * sqrt(3.0 * omz);
        int64_t jp = (int64_t)(tp * tmp), jm = (int64_t)((1.0 - tp) * tmp);
        if (jp > nside - 1) jp = nside - 1;
        if (jm > nside - 1) jm = nside - 1;
        if (z >= 0.0) { face = ntt; ix = nside - jm - 1; iy = nside - jp - 1; }
        else { face = ntt + 8; ix = jp; iy = jm; }
    }
    return face * nside * nside + spread_bits(ix) + 2 * spread_bits(iy);
}

/* Children of a merged "vertex" ray (reading of Sec. 3.2-3.3).  A merged ray
 * points along the centre of merge pixel pm (level lm) and carries level
 * l >= lm.  In the NESTED scheme the centre of a pixel is the corner shared
 * by its four children, and at every deeper level by exactly four pixels:
 * descend into child i, then always into the sub-pixel 3-i that touches that
 * corner.  These four level-(l+1) pixels tile the solid angle of one level-l
 * pixel around the merged direction and are its split children; child
 * c = i*4^(m-1) + j of an m-level split is their descendant j. */
int64_t or_vertex_child(int lm, int64_t pm, int l, int m, int64_t c)
{
    const int depth = l + 1 - lm;                   /* >= 1 */
    const int64_t i = c >> (2 * (m - 1)), j = c & (((int64_t)1 << (2 * (m - 1))) - 1);
    int64_t q = pm * 4 + i;
    for (int k = 1; k < depth; ++k) q = q * 4 + (3 - i);
    return (q << (2 * (m - 1))) + j;
}

/* ------------------------------------------------------------------------- */
int or_traverse(const int64_t p0[3], const int32_t d[3], const int32_t n[3],
                int32_t cells[4][3], double ds[4], int *escaped)
{
    int64_t cell[3], D[3], ad[3];
    int sg[3];
    for (int a = 0; a < 3; ++a) {
        ad[a] = d[a] < 0 ? -(int64_t)d[a] : (int64_t)d[a];
        sg[a] = d[a] > 0 ? 1 : (d[a] < 0 ? -1 : 0);
        if (d[a] > 0) {
            cell[a] = floordiv64(p0[a], OR_S);
            D[a] = (cell[a] + 1) * OR_S - p0[a];
        } else if (d[a] < 0) {
            cell[a] = floordiv64(p0[a] - 1, OR_S);
            D[a] = p0[a] - cell[a] * OR_S;
        } else {
            cell[a] = floordiv64(p0[a], OR_S);
            D[a] = 0;
        }
    }
    int64_t tn = 0, td = 1; /* start of the current segment, t = tn/td */
    int nseg = 0;
    *escaped = 0;
    for (;;) {
        for (int a = 0; a < 3; ++a)
            if (cell[a] < 0 || cell[a] >= n[a]) { *escaped = 1; return nseg; }
        int amin = -1;
        for (int a = 0; a < 3; ++a) {
            if (sg[a] == 0 || D[a] >= ad[a]) continue;  /* no crossing before t=1 */
            if (amin < 0 || D[a] * ad[amin] < D[amin] * ad[a]) amin = a;
        }
        int64_t un, ud;
        if (amin < 0) { un = 1; ud = 1; }
        else { un = D[amin]; ud = ad[amin]; }
        /* ds = un/ud - tn/td, numerator exact in int64 */
        int64_t num = un * td - tn * ud, den = ud * td;
        if (nseg >= 4) return -1; /* cannot happen for |d_a| <= 2^21 */
        cells[nseg][0] = (int32_t)cell[0];
        cells[nseg][1] = (int32_t)cell[1];
        cells[nseg][2] = (int32_t)cell[2];
        ds[nseg] = (double)num / (double)den;
        nseg++;
        if (amin < 0) return nseg;
        int64_t Dm = D[amin], am = ad[amin];
        for (int a = 0; a < 3; ++a) {
            if (sg[a] == 0 || D[a] >= ad[a]) continue;
            if (D[a] * am == Dm * ad[a]) { cell[a] += sg[a]; D[a] += OR_S; }
        }
        tn = Dm; td = am;
    }
}

/* ------------------------------------------------------------------------- */
/* Rate coefficients.                                                         */
/* Sec. 4.1 cites Hui & Gnedin (1997) for the thermal solution; their fits    */
/* (their Appendix, lambda = 2*157807 K / T) are used for alpha_B, case-B     */
/* recombination cooling and collisional ionisation; collisional excitation   */
/* and free-free cooling follow Cen (1992); Compton cooling off the CMB is    */
/* written from physical constants.                                           */
/* ------------------------------------------------------------------------- */
static const double KB = 1.380649e-16;       /* erg/K */
static const double T_HI = 157807.0;         /* K     */
static const double EV = 1.602176634e-12;    /* erg   */

double or_alpha_B(double T)
{
    double lam = 2.0 * T_HI / T;
    return 2.753e-14 * pow(lam, 1.5) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
}
/* case-A recombination coefficient (Hui & Gnedin 1997), cm^3/s */
double or_alpha_A(double T)
{
    double lam = 2.0 * T_HI / T;
    return 1.269e-13 * pow(lam, 1.503) / pow(1.0 + pow(lam / 0.522, 0.470), 1.923);
}

/* Mean energy given to the gas per HI photo-ionisation for a power-law
 * spectrum J ~ nu^-alpha cut off at 4 Ryd with sigma ~ nu^-beta, beta = 2.75
 * (the bracket of Sec. 4.2, Eq. 22), erg */
double or_pl_heat_per_ion(double alpha_pl)
{
    const double a = alpha_pl + 2.75;
    return 13.6 * EV * (a / (a - 1.0) * (1.0 - pow(4.0, 1.0 - a)) / (1.0 - pow(4.0, -a)) - 1.0);
}

double or_coll_ion(double T)
{
    double lam = 2.0 * T_HI / T;
    return 21.11 * pow(T, -1.5) * exp(-lam / 2.0) * pow(lam, -1.089) /
           pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
}
/* net cooling rate Lambda (erg s^-1 cm^-3) */
double or_cooling(double T, double ne, double nHI, double nHII, double z)
{
    double lam = 2.0 * T_HI / T;
    double rec = 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
    double cion = 13.6 * EV * or_coll_ion(T);
    double cexc = 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1.0e5));
    double lt = log10(T);
    double gff = 1.1 + 0.34 * exp(-(5.5 - lt) * (5.5 - lt) / 3.0);
    double ff = 1.42e-27 * gff * sqrt(T);
    /* Compton: 4 k_B sigma_T a T_cmb^4 (T - T_cmb) n_e / (m_e c) */
    const double sigma_T = 6.6524587e-25, a_rad = 7.5657e-15, m_e = 9.1093837e-28, c = 2.99792458e10;
    double Tc = 2.7255 * (1.0 + z);
    double comp = 4.0 * KB * sigma_T * a_rad * Tc * Tc * Tc * Tc / (m_e * c) * (T - Tc);
    return rec * ne * nHII + cion * ne * nHI + cexc * ne * nHI + ff * ne * nHII + comp * ne;
}

/* ------------------------------------------------------------------------- */
/* One cell's ionisation update (Sec. 4.1, Eq. 6-10) at fixed Gamma:          */
/* x(t) = x_eq + (x0 - x_eq) exp(-t/t_i), <x> its average over dt, with n_e   */
/* re-evaluated from <x> `iters` times.  Written for the neutral fraction     */
/* y = 1 - x: y_eq = alpha n_e / (Gamma + C n_e + alpha n_e).                 */
/* ------------------------------------------------------------------------- */
void or_chem_cell(double nH, double G, double alpha, double C, double dt, int iters,
                  double y0, double *y1_out, double *ybar_out)
{
    double ybar = y0, y1 = y0;
    for (int it = 0; it < iters; ++it) {
        double ne = nH * (1.0 - ybar);
        double a = G + C * ne, b = alpha * ne;
        double sum = a + b;
        if (!(sum > 0.0)) { y1 = y0; ybar = y0; break; }
        double yeq = b / sum;
        double r = dt * sum; /* dt / t_i */
        y1 = yeq + (y0 - yeq) * exp(-r);
        ybar = yeq + (y0 - yeq) * (-expm1(-r)) / r;
    }
    *y1_out = y1;
    *ybar_out = ybar;
}

/* Temperature update (Sec. 4.1, Eq. 12 with H(z) = 0 and static density):
 * the particle-number term first, T n_tot conserved over the step; then the
 * radiative term 2/(3 k n_tot) (H - Lambda) by explicit sub-steps of at most
 * 5% of T, at most 1000 of them. */
double or_temperature(double T, double nH, double x0, double x1, double xbar,
                      double heat, double z, double dt)
{
    T = T * (1.0 + x0) / (1.0 + x1);
    double ne = nH * xbar, nHII = nH * xbar, nHI = nH * (1.0 - xbar), ntot = nH * (1.0 + xbar);
    double left = dt;
    for (int k = 0; k < 1000 && left > 0.0; ++k) {
        double dTdt = 2.0 / (3.0 * KB * ntot) * (heat - or_cooling(T, ne, nHI, nHII, z));
        double h = left;
        if (k < 999 && dTdt != 0.0) {
            double lim = 0.05 * T / fabs(dTdt);
            if (lim < h) h = lim;
        }
        T += dTdt * h;
        left -= h;
    }
    return T;
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t l;       /* HEALPix level                */
    int64_t p;       /* NESTED pixel                 */
    int32_t e;       /* emitter (source cell); merged rays: local cell of the merge */
    int32_t b;       /* birth step; merged rays: step of the merge  */
    int32_t d[3];    /* fixed-point direction        */
    double N[OR_MAXB]; /* photons per bin            */
    /* merged rays (Sec. 3.3) and their split children only */
    int32_t kind;    /* 0 cast by an emitter, 1 made by a merge           */
    int32_t vflag;   /* 1: unsplit merged ray of level l > l_merge, centred
                        on the vertex shared by its four level-(l+1) children
                        (p is then the level-l_merge merge pixel)         */
    int32_t A;       /* distance travelled at the merge, in cells         */
    int64_t P[3];    /* position at the merge (fixed point)               */
    double thr;      /* termination threshold, photons                    */
} or_ray;

typedef struct {
    int32_t nx, ny, nz;
    double dx;          /* physical cell size, cm      */
    double z;           /* redshift (fixed)            */
    int32_t nb;
    double frac[OR_MAXB], sigma[OR_MAXB], eheat[OR_MAXB];
    int32_t mfp_mode;   /* 0 none, 1 constant lambda, 2 power law in ionised cells */
    double lambda0_c, delta_exp, gamma_ref, gamma_exp, gamma_floor, xion_thr, nH_mean;
    int32_t l_src, l_max;
    double n_min, eps_term;
    uint64_t seed;
    int32_t rotate, isothermal, rates, chem_iters;
    double alpha_const, x_init, T_init;
    int32_t merge, l_merge;   /* ray merging on/off, level of the merge sphere */
    double n_ex;              /* rays exempt from merging per RT cell          */
    int32_t gamma_iters;      /* passes of the Gamma - <n_HI> iteration (>= 1)  */
    int32_t gen_mode;         /* 1: Generalized Opacity mode (Sec. 4.2)        */
    double chi;               /* He/H number ratio of Eq. 18 (singly ionised He) */
    double t_reion;           /* Generalized mode: temperature of newly ionised gas (K) */
    double alpha_pl;          /* Generalized mode: spectral index of Eq. 22's heating   */
} or_config;

typedef struct {
    or_config c;
    int64_t ncell;
    double *nH, *y, *T, *gamma, *kap_sub;  /* per cell state; kap_sub in cm^-1 */
    double *ion, *heat, *absd;            /* per step accumulators           */
    double *y_est, *k_est;                /* iteration: <y> and sub-grid opacity */
    double *xion, *yion, *front, *fall, *rho;   /* Generalized mode: ionised volume fraction,
                                             neutral fraction inside it, photons the screen
                                             absorbed / that reached it this pass, and the
                                             fraction of arriving photons it absorbs */
    int32_t *segcnt;                      /* segments per cell, last step    */
    int32_t K[OR_MAXL];
    /* emitters */
    int32_t ne, ecap;
    int32_t *ecell;                       /* 3 per emitter                   */
    double *endot;
    /* rays */
    or_ray *rays;
    int64_t nray, rcap;
    int64_t step;
    double emitted, absorbed, escaped, in_flight;
    int64_t segments_total, segments_last, near_threshold;
} or_sim;

static int grow_rays(or_ray **buf, int64_t *cap, int64_t need)
{
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    or_ray *nb = (or_ray *)realloc(*buf, (size_t)nc * sizeof(or_ray));
    if (!nb) return -1;
    *buf = nb;
    *cap = nc;
    return 0;
}

/* Sub-grid opacity (cm^-1) of cell i for neutral fraction y and photo-
 * ionisation rate G (Sec. 4.2, the lambda law of the configuration) */
static double kappa_sub_of(const or_sim *S, int64_t i, double y, double G)
{
    const or_config *c = &S->c;
    double k = 0.0;
    if (c->mfp_mode == 1) {
        k = (1.0 + c->z) / c->lambda0_c;
    } else if (c->mfp_mode == 2 && c->gen_mode) {
        /* the ionised component; a cell never lit yet is optically thin
         * (the Eq. 14 guess) */
        if (G > 0.0) {
            double delta = S->nH[i] / c->nH_mean;
            double g = G > c->gamma_floor ? G : c->gamma_floor;
            k = (1.0 + c->z) / (c->lambda0_c * pow(delta, -c->delta_exp) * pow(g / c->gamma_ref, c->gamma_exp));
        }
    } else if (c->mfp_mode == 2) {
        if (1.0 - y >= c->xion_thr) {
            double delta = S->nH[i] / c->nH_mean;
            double g = G > c->gamma_floor ? G : c->gamma_floor;
            double lam_c = c->lambda0_c * pow(delta, -c->delta_exp) * pow(g / c->gamma_ref, c->gamma_exp);
            k = (1.0 + c->z) / lam_c;
        }
    }
    return k;
}

/* Generalized mode, neutral fraction of the highly ionised component: with
 * the equilibrium model (mfp mode 3, Eq. 20-22) n_HI = alpha n_e n_HII /
 * Gamma = alpha (1 + chi) n_H^2 / Gamma; a cell never lit yet (Gamma = 0) is
 * optically thin (the Eq. 14 guess); other laws carry their opacity in
 * kappa_sub. */
static double gen_y_ion(const or_sim *S, int64_t i, double G)
{
    const or_config *c = &S->c;
    if (c->mfp_mode != 3 || !(G > 0.0)) return 0.0;
    double alpha = c->rates ? or_alpha_B(S->T[i]) : c->alpha_const;
    double g = G > c->gamma_floor ? G : c->gamma_floor;
    double y = alpha * (1.0 + c->chi) * S->nH[i] / g;
    return y < 1.0 ? y : 1.0;
}

/* Generalized mode, temperature of the ionised gas (Sec. 4.2): newly
 * ionised gas enters at T_reion and mixes by mass with the gas already
 * ionised; then Eq. 12 (static density) with the photo-heating of Eq. 22 --
 * photo-ionisation equilibrium, so each recombination (case A) is one
 * ionisation bringing the power-law mean excess energy -- against the
 * cooling rates, with n_HI from the ionised part's neutral fraction and
 * n_e = n_HII + chi n_H (singly ionised helium).
 * Sub-steps are the two-stage Rosenbrock scheme ROS2 (Verwer, Spee, Blom
 * & Hundsdorfer 1999; gamma = 1 + 1/sqrt 2), second order whatever the
 * Jacobian used: here f' from a one-sided difference over 10^-3 T, taken
 * as 0 where it is positive.  Each sub-step is at most the one that would
 * change T by 5% explicitly (at most 1000 sub-steps, the last takes what is
 * left); the scheme is L-stable, so a step far longer than the time the gas
 * takes to reach its equilibrium temperature ends at that temperature. */
static double gen_dTdt(double T, double nHI, double nHII, double ne, double ntot, double epl, double z)
{
    const double heat = epl * or_alpha_A(T) * ne * nHII;
    return 2.0 / (3.0 * KB * ntot) * (heat - or_cooling(T, ne, nHI, nHII, z));
}

double or_gen_temperature(double T, double x0, double x1, double yion, double nH, double chi, double t_reion,
                          double alpha_pl, double z, double dt)
{
    if (x1 > x0) T = (x0 * T + (x1 - x0) * t_reion) / x1;
    const double nHII = nH * (1.0 - yion), nHI = nH * yion, ne = nHII + chi * nH;
    const double ntot = nH * (1.0 + chi) + ne;
    const double epl = or_pl_heat_per_ion(alpha_pl);
    double left = dt;
    const double g = 1.0 + 1.0 / sqrt(2.0);
    for (int k = 0; k < 1000 && left > 0.0; ++k) {
        const double f = gen_dTdt(T, nHI, nHII, ne, ntot, epl, z);
        if (f == 0.0) break;
        double J = (gen_dTdt(T * 1.001, nHI, nHII, ne, ntot, epl, z) - f) / (0.001 * T);
        if (J > 0.0) J = 0.0;
        double h = left;
        if (k < 999) {
            double lim = 0.05 * T / fabs(f);
            if (lim < h) h = lim;
        }
        const double w = 1.0 / (1.0 - g * h * J);
        const double k1 = w * f;
        const double k2 = w * (gen_dTdt(T + h * k1, nHI, nHII, ne, ntot, epl, z) - 2.0 * k1);
        T += h * (1.5 * k1 + 0.5 * k2);
        left -= h;
    }
    return T;
}

static double gen_temperature(const or_sim *S, int64_t i, double x0, double x1, double yion, double dt)
{
    const or_config *c = &S->c;
    return or_gen_temperature(S->T[i], x0, x1, yion, S->nH[i], c->chi, c->t_reion, c->alpha_pl, c->z, dt);
}

static void update_kappa_sub(or_sim *S, int64_t i)
{
    S->kap_sub[i] = kappa_sub_of(S, i, S->y[i], S->gamma[i]);
}

or_sim *or_create(const or_config *cfg, const double *nH)
{
    or_sim *S = (or_sim *)calloc(1, sizeof(or_sim));
    if (!S) return NULL;
    S->c = *cfg;
    S->ncell = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    int64_t n = S->ncell;
    S->nH = malloc(n * sizeof(double));
    S->y = malloc(n * sizeof(double));
    S->T = malloc(n * sizeof(double));
    S->gamma = calloc(n, sizeof(double));
    S->kap_sub = calloc(n, sizeof(double));
    S->ion = calloc(n, sizeof(double));
    S->heat = calloc(n, sizeof(double));
    S->absd = calloc(n, sizeof(double));
    S->segcnt = calloc(n, sizeof(int32_t));
    S->y_est = calloc(n, sizeof(double));
    S->k_est = calloc(n, sizeof(double));
    S->xion = calloc(n, sizeof(double));
    S->yion = calloc(n, sizeof(double));
    S->front = calloc(n, sizeof(double));
    S->fall = calloc(n, sizeof(double));
    S->rho = malloc(n * sizeof(double));
    if (!S->nH || !S->y || !S->T || !S->gamma || !S->kap_sub || !S->ion || !S->heat || !S->absd || !S->segcnt ||
        !S->y_est || !S->k_est || !S->xion || !S->yion || !S->front || !S->fall || !S->rho)
        return NULL;
    if (S->c.nH_mean <= 0.0) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += nH[i];
        S->c.nH_mean = s / (double)n;
    }
    for (int64_t i = 0; i < n; ++i) {
        S->nH[i] = nH[i];
        S->y[i] = cfg->gen_mode ? 1.0 : 1.0 - cfg->x_init;   /* Generalized mode: no ionised fraction yet */
        S->rho[i] = 1.0;
        S->T[i] = cfg->T_init;
        update_kappa_sub(S, i);
    }
    or_split_table(cfg->n_min, S->K);
    return S;
}

void or_destroy(or_sim *S)
{
    if (!S) return;
    free(S->nH); free(S->y); free(S->T); free(S->gamma); free(S->kap_sub);
    free(S->ion); free(S->heat); free(S->absd); free(S->segcnt); free(S->y_est); free(S->k_est);
    free(S->xion); free(S->yion); free(S->front); free(S->fall); free(S->rho);
    free(S->ecell); free(S->endot); free(S->rays);
    free(S);
}

/* Sources in one cell form one emitter (Sec. 3.1: rays are cast from each
 * cell that contains sources); emitters are numbered in order of the first
 * source seen in their cell, and their rates add. */
int or_add_sources(or_sim *S, int32_t n, const int32_t *ijk, const double *ndot)
{
    for (int32_t s = 0; s < n; ++s) {
        const int32_t *q = ijk + 3 * s;
        if (q[0] < 0 || q[0] >= S->c.nx || q[1] < 0 || q[1] >= S->c.ny || q[2] < 0 || q[2] >= S->c.nz)
            return -1;
        int found = -1;
        for (int32_t e = 0; e < S->ne; ++e)
            if (S->ecell[3 * e] == q[0] && S->ecell[3 * e + 1] == q[1] && S->ecell[3 * e + 2] == q[2]) { found = e; break; }
        if (found >= 0) { S->endot[found] += ndot[s]; continue; }
        if (S->ne == S->ecap) {
            int32_t nc = S->ecap ? 2 * S->ecap : 16;
            int32_t *c2 = realloc(S->ecell, (size_t)nc * 3 * sizeof(int32_t));
            double *n2 = realloc(S->endot, (size_t)nc * sizeof(double));
            if (!c2 || !n2) return -2;
            S->ecell = c2; S->endot = n2; S->ecap = nc;
        }
        S->ecell[3 * S->ne] = q[0];
        S->ecell[3 * S->ne + 1] = q[1];
        S->ecell[3 * S->ne + 2] = q[2];
        S->endot[S->ne] = ndot[s];
        S->ne++;
    }
    return 0;
}

/* Deposit the photons a ray still carries into `cell` as if the ray stayed
 * there for ever (termination; reading of Sec. 2.1's "rays disappear when
 * tau >> 1": the leftover is absorbed where the ray stops). */
static void deposit_all(or_sim *S, int64_t cell, const double *N, const double *kap, double *absorbed)
{
    const or_config *c = &S->c;
    for (int b = 0; b < c->nb; ++b) {
        S->absd[cell] += N[b];
        *absorbed += N[b];
        if (kap[b] > 0.0) {
            S->ion[cell] += c->sigma[b] * N[b] / kap[b];
            S->heat[cell] += c->eheat[b] * c->sigma[b] * N[b] / kap[b];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Ray merging at the end of a step (Sec. 3.3, Eq. 4)                         */
/* ------------------------------------------------------------------------- */
/* Readings where the section is silent:
 *  - rank: a ray's photon content is the sum of its bins; with
 *    K = floor(N_ex * N_RT), every ray whose content is at least the K-th
 *    largest, T_ref, is exempt (ties at the K-th value are all exempt; K = 0
 *    exempts nothing; K >= the number of rays merges nothing);
 *  - cell: the cell holding the ray's end point (floor per axis); a ray whose
 *    end point is on the far face of the box is not merged;
 *  - sphere: one random rotation per (cell, step), drawn like an emitter's
 *    (or_merge_rotation);
 *  - merged ray: photons summed per bin; position, distance travelled and
 *    HEALPix level are the photon-weighted means of the constituents'
 *    (weight: the ray's content), each rounded once to nearest (the
 *    fixed-point grid, whole cells, whole levels; the level at least
 *    l_merge); direction the centre of the merge pixel; termination threshold
 *    the sum of the constituents'.  A group of one ray keeps the ray. */
typedef struct { int64_t key, idx; } or_mkey;

static int cmp_mkey(const void *a, const void *b)
{
    const or_mkey *x = (const or_mkey *)a, *y = (const or_mkey *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int cmp_double_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return x > y ? -1 : (x < y);
}

static int or_merge(or_sim *S, double dt, int64_t s, int64_t Kin)
{
    const or_config *c = &S->c;
    const int64_t n = S->nray;
    const double Kd = Kin >= 0 ? (double)Kin : floor(c->n_ex * (double)S->ncell);
    if (Kd >= (double)n) return 0;
    const int64_t K = (int64_t)Kd;
    const int64_t ncast = 12LL << (2 * c->l_src);
    const int64_t ndir = 12LL << (2 * c->l_merge);
    double *T = malloc((size_t)n * sizeof(double)), *Ts = malloc((size_t)n * sizeof(double));
    or_mkey *mk = malloc((size_t)n * sizeof(or_mkey));
    int64_t (*p1) = malloc((size_t)n * 3 * sizeof(int64_t));
    char *dead = calloc((size_t)n, 1);
    if (!T || !Ts || !mk || !p1 || !dead) return -1;
    /* rank by photon content (Sec. 3.3: "rank-ordered by the number of
     * photons they contain") */
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int b = 0; b < c->nb; ++b) t += S->rays[i].N[b];
        Ts[i] = T[i] = t;
    }
    double Tstar = INFINITY;
    if (K > 0) {
        qsort(Ts, (size_t)n, sizeof(double), cmp_double_desc);
        Tstar = Ts[K - 1];
    }
    int64_t nm = 0;
    const int64_t nn[3] = {c->nx, c->ny, c->nz};
    for (int64_t i = 0; i < n; ++i) {
        const or_ray *r = &S->rays[i];
        if (T[i] >= Tstar) continue;                        /* exempt */
        int64_t *q = p1 + 3 * i, cell[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            if (r->kind == 0) q[a] = (2 * (int64_t)S->ecell[3 * r->e + a] + 1) * (OR_S / 2) + (s - r->b + 1) * (int64_t)r->d[a];
            else q[a] = r->P[a] + (s - r->b) * (int64_t)r->d[a];
            cell[a] = floordiv64(q[a], OR_S);
            if (cell[a] < 0 || cell[a] >= nn[a]) inside = 0;
        }
        if (!inside) continue;
        int64_t local = (cell[2] * c->ny + cell[1]) * c->nx + cell[0];
        int32_t Rq[9];
        or_merge_rotation(c->seed, local, s, c->rotate, Rq);
        mk[nm].key = local * ndir + or_merge_pixel(c->l_merge, Rq, r->d);
        mk[nm].idx = i;
        nm++;
    }
    qsort(mk, (size_t)nm, sizeof(or_mkey), cmp_mkey);
    or_ray *merged = NULL;
    int64_t nmerged = 0, mcap = 0;
    for (int64_t g0 = 0; g0 < nm;) {
        int64_t g1 = g0 + 1;
        while (g1 < nm && mk[g1].key == mk[g0].key) g1++;
        if (g1 - g0 >= 2) {
            or_ray m;
            memset(&m, 0, sizeof(m));
            const int64_t local = mk[g0].key / ndir, pm = mk[g0].key % ndir;
            const int64_t cell[3] = {local % c->nx, (local / c->nx) % c->ny, local / ((int64_t)c->nx * c->ny)};
            /* photon-weighted sums; positions relative to the cell's corner */
            double W = 0.0, wp[3] = {0.0, 0.0, 0.0}, wa = 0.0, wl = 0.0, thr = 0.0;
            for (int64_t k = g0; k < g1; ++k) {
                const int64_t i = mk[k].idx;
                const or_ray *r = &S->rays[i];
                const double w = T[i];
                for (int b = 0; b < c->nb; ++b) m.N[b] += r->N[b];
                for (int a = 0; a < 3; ++a) wp[a] += w * (double)(p1[3 * i + a] - cell[a] * OR_S);
                const int64_t dist = r->kind == 0 ? s - r->b + 1 : r->A + (s - r->b);
                wa += w * (double)dist;
                wl += w * (double)r->l;
                thr += r->kind == 0 ? c->eps_term * S->endot[r->e] * dt / (double)ncast * ldexp(1.0, -2 * (r->l - c->l_src))
                                    : r->thr;
                W += w;
                dead[i] = 1;
            }
            for (int a = 0; a < 3; ++a) {
                int64_t v = W > 0.0 ? (int64_t)nearbyint(wp[a] / W) : 0;
                if (v < 0) v = 0;
                if (v > OR_S - 1) v = OR_S - 1;
                m.P[a] = cell[a] * OR_S + v;
            }
            const double Am = W > 0.0 ? nearbyint(wa / W) : 0.0;
            m.A = (int32_t)(Am < 0.0 ? 0.0 : (Am > 65535.0 ? 65535.0 : Am));
            int64_t L = W > 0.0 ? (int64_t)nearbyint(wl / W) : c->l_merge;
            if (L < c->l_merge) L = c->l_merge;
            if (L > c->l_max) L = c->l_max;
            m.l = (int32_t)L;
            m.p = pm;
            m.kind = 1;
            m.vflag = L > c->l_merge;
            m.e = (int32_t)local;
            m.b = (int32_t)s;
            m.thr = thr;
            int32_t Rq[9];
            or_merge_rotation(c->seed, local, s, c->rotate, Rq);
            or_direction(c->l_merge, pm, Rq, m.d);
            if (grow_rays(&merged, &mcap, nmerged + 1)) return -1;
            merged[nmerged++] = m;
        }
        g0 = g1;
    }
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i)
        if (!dead[i]) S->rays[w++] = S->rays[i];
    if (grow_rays(&S->rays, &S->rcap, w + nmerged)) return -1;
    for (int64_t k = 0; k < nmerged; ++k) S->rays[w++] = merged[k];
    S->nray = w;
    free(T); free(Ts); free(mk); free(p1); free(dead); free(merged);
    return 0;
}

/* One march of every live ray by one cell width (Sec. 3.1) with absorption
 * (Eq. 13, 17), escape, termination and splits, through the opacities of
 * neutral fraction yk and sub-grid opacity ksub (cm^-1) per cell.  Fills the
 * per-cell deposits and returns the surviving rays and children in *out; the
 * photon tallies go to *t.  The live rays themselves are not changed. */
typedef struct { double absorbed, escaped; int64_t segs, near; } or_tally;

static int or_march(or_sim *S, double dt, const double *yk, const double *ksub, or_ray **out_p, int64_t *nout_p,
                    int64_t *ocap_p, or_tally *t)
{
    const or_config *c = &S->c;
    const int32_t n3[3] = {c->nx, c->ny, c->nz};
    const int64_t ncast = 12LL << (2 * c->l_src);
    const int64_t s = S->step;
    memset(t, 0, sizeof(*t));
    for (int64_t i = 0; i < S->ncell; ++i) {
        S->ion[i] = 0.0; S->heat[i] = 0.0; S->absd[i] = 0.0; S->segcnt[i] = 0; S->front[i] = 0.0; S->fall[i] = 0.0;
    }
    or_ray *out = NULL;
    int64_t nout = 0, ocap = 0;
    for (int64_t ir = 0; ir < S->nray; ++ir) {
        or_ray r = S->rays[ir];
        /* age: distance travelled before this step, in cells.  A ray cast by
         * an emitter starts at the emitter's cell centre; a merged ray at its
         * merge position, with the distance its constituents had travelled */
        int64_t age, p0[3];
        if (r.kind == 0) {
            age = s - r.b;
            const int32_t *ec = S->ecell + 3 * r.e;
            for (int a = 0; a < 3; ++a) p0[a] = (2 * (int64_t)ec[a] + 1) * (OR_S / 2) + age * (int64_t)r.d[a];
        } else {
            int64_t since = s - r.b - 1;
            age = r.A + since;
            for (int a = 0; a < 3; ++a) p0[a] = r.P[a] + since * (int64_t)r.d[a];
        }
        int32_t cells[4][3];
        double ds[4];
        int esc;
        int ns = or_traverse(p0, r.d, n3, cells, ds, &esc);
        if (ns < 0) return -3;
        int64_t last = -1;
        double kap[OR_MAXB];
        int screened = 0;
        for (int k = 0; k < ns && !screened; ++k) {
            int64_t ci = ((int64_t)cells[k][2] * c->ny + cells[k][1]) * c->nx + cells[k][0];
            double nHI = S->nH[ci] * yk[ci];
            double dsp = ds[k] * c->dx; /* path length, cm */
            /* Generalized mode (Sec. 4.2, Eq. 19): the ray crosses the ionised
             * fraction x_ion of its path with the sub-grid opacity; what then
             * reaches the neutral rest stops at the screen (Eq. 18) */
            const double xg = c->gen_mode ? S->xion[ci] : 1.0;
            if (c->gen_mode) dsp *= xg;
            for (int b = 0; b < c->nb; ++b) {
                kap[b] = nHI * c->sigma[b] + ksub[ci];
                double tau = kap[b] * dsp;
                double absb = -r.N[b] * expm1(-tau); /* N (1 - e^-tau) */
                /* Eq. 17: N (1 - e^{-ds/lambda}) sigma lambda, lambda = 1/kappa */
                double ion = kap[b] > 0.0 ? c->sigma[b] * absb / kap[b] : c->sigma[b] * r.N[b] * dsp;
                S->ion[ci] += ion;
                S->heat[ci] += c->eheat[b] * ion;
                S->absd[ci] += absb;
                t->absorbed += absb;
                r.N[b] = r.N[b] * exp(-tau);
            }
            S->segcnt[ci] += 1;
            last = ci;
            if (xg < 1.0) {
                /* the screen absorbs the fraction rho of what reaches it (all of
                 * it while the cell has atoms to spare); the rest crosses the
                 * gas the front ionises during the step and goes on */
                const double rh = S->rho[ci];
                double nf = 0.0;
                for (int b = 0; b < c->nb; ++b) {
                    nf += r.N[b];
                    r.N[b] = rh >= 1.0 ? 0.0 : r.N[b] * (1.0 - rh);
                }
                S->fall[ci] += nf;
                S->front[ci] += rh * nf;
                t->absorbed += rh * nf;
                if (rh >= 1.0) {
                    t->segs += k + 1;
                    screened = 1;
                }
            }
        }
        if (screened) continue;
        t->segs += ns;
        if (esc) {
            for (int b = 0; b < c->nb; ++b) t->escaped += r.N[b];
            continue;
        }
        /* termination: below eps of the ray's unattenuated content */
        double tot = 0.0;
        for (int b = 0; b < c->nb; ++b) tot += r.N[b];
        double thr = r.kind == 0 ? c->eps_term * S->endot[r.e] * dt / (double)ncast * ldexp(1.0, -2 * (r.l - c->l_src))
                                 : r.thr;
        if (fabs(tot - thr) <= 1e-4 * thr) t->near++;
        if (tot < thr) {
            deposit_all(S, last, r.N, kap, &t->absorbed);
            continue;
        }
        /* splitting (Sec. 3.2, Eq. 2-3): the ray has travelled age+1 cells */
        int m = 0;
        while (r.l + m < c->l_max && age + 1 >= S->K[r.l + m]) m++;
        int64_t nchild = (int64_t)1 << (2 * m);
        if (grow_rays(&out, &ocap, nout + nchild)) return -2;
        if (m == 0) { out[nout++] = r; continue; }
        /* children keep the rotation of their parent's sphere (Sec. 3.2):
         * the emitter's at the birth step, or the merge cell's at the merge */
        double R[9];
        int32_t Rq[9];
        if (r.kind == 0) or_rotation(c->seed, r.e, r.b, c->rotate, R, Rq);
        else or_merge_rotation(c->seed, r.e, r.b, c->rotate, Rq);
        for (int64_t j = 0; j < nchild; ++j) {
            or_ray ch = r;
            ch.l = r.l + m;
            ch.p = r.vflag ? or_vertex_child(c->l_merge, r.p, r.l, m, j) : r.p * nchild + j;
            ch.vflag = 0;
            ch.thr = r.thr / (double)nchild;
            or_direction(ch.l, ch.p, Rq, ch.d);
            for (int b = 0; b < c->nb; ++b) ch.N[b] = r.N[b] / (double)nchild;
            out[nout++] = ch;
        }
    }
    *out_p = out; *nout_p = nout; *ocap_p = ocap;
    return 0;
}

/* Chemistry and temperature per cell (Sec. 4.1) from this step's deposits.
 * final = 0: one pass of the Gamma - <n_HI> iteration (Eq. 7-11; with the
 * sub-grid law also the lambda - Gamma iteration of Sec. 4.2): the state is
 * left unchanged, and y_est / ksub_est receive the time-averaged neutral
 * fraction and the sub-grid opacity the next march uses.  final = 1: the
 * step's update is committed. */
static void or_chem(or_sim *S, double dt, int final, double *y_est, double *ksub_est)
{
    const or_config *c = &S->c;
    const double V = c->dx * c->dx * c->dx;
    if (c->gen_mode) {
        /* Generalized mode: Gamma of the ionised component (Eq. 17 with
         * ds -> x_ion ds and V -> x_ion V); the screen advances by the photons
         * it absorbed over the atoms it ionises (Eq. 18), the ionised part
         * loses what recombines beyond its absorptions; temperature as
         * gen_temperature (or fixed when isothermal).  The
         * screen's share of arriving photons for the next pass (or step) is
         * the atoms it has left over the photons that reached it */
        for (int64_t i = 0; i < S->ncell; ++i) {
            const double x = S->xion[i];
            const double G = x > 0.0 ? S->ion[i] / (x * V * dt) : 0.0;
            const double A = (1.0 + c->chi) * S->nH[i] * V;      /* atoms of a whole cell */
            if (!final) {
                y_est[i] = gen_y_ion(S, i, G);
                ksub_est[i] = kappa_sub_of(S, i, 0.0, G);
                S->rho[i] = S->fall[i] > (1.0 - x) * A ? (1.0 - x) * A / S->fall[i] : 1.0;
                continue;
            }
            /* net atom balance of the cell: photons absorbed at the screen and
             * in the ionised part, minus recombinations in the ionised part
             * (alpha (1 + chi) n_H^2 x V dt, the approximation of Eq. 22); in
             * photo-ionisation equilibrium the last two cancel and this is Eq. 18 */
            const double alpha = c->rates ? or_alpha_B(S->T[i]) : c->alpha_const;
            const double rec = alpha * (1.0 + c->chi) * S->nH[i] * S->nH[i] * x * V * dt;
            double x1 = x + (S->front[i] + S->absd[i] - rec) / A;
            if (x1 > 1.0) x1 = 1.0;
            if (x1 < 0.0) x1 = 0.0;
            S->rho[i] = S->fall[i] > (1.0 - x1) * A ? (1.0 - x1) * A / S->fall[i] : 1.0;
            if (!c->isothermal && x1 > 0.0)
                S->T[i] = gen_temperature(S, i, x, x1, gen_y_ion(S, i, G), dt);
            S->xion[i] = x1;
            S->gamma[i] = G;
            S->yion[i] = gen_y_ion(S, i, G);
            S->kap_sub[i] = kappa_sub_of(S, i, 0.0, G);
            S->y[i] = (1.0 - x1) + x1 * S->yion[i];
        }
        return;
    }
    for (int64_t i = 0; i < S->ncell; ++i) {
        double G = S->ion[i] / (V * dt);     /* Eq. 17 */
        double Hn = S->heat[i] / (V * dt);   /* sum_nu E_nu Gamma_nu */
        double T0 = S->T[i];
        double alpha = c->rates ? or_alpha_B(T0) : c->alpha_const;
        double C = c->rates ? or_coll_ion(T0) : 0.0;
        double y0 = S->y[i], y1, ybar;
        or_chem_cell(S->nH[i], G, alpha, C, dt, c->chem_iters, y0, &y1, &ybar);
        if (!final) {
            y_est[i] = ybar;
            ksub_est[i] = kappa_sub_of(S, i, ybar, G);
            continue;
        }
        if (!c->isothermal) {
            double heat = S->nH[i] * ybar * Hn;
            S->T[i] = or_temperature(T0, S->nH[i], 1.0 - y0, 1.0 - y1, 1.0 - ybar, heat, c->z, dt);
        }
        S->y[i] = y1;
        S->gamma[i] = G;
        update_kappa_sub(S, i);
    }
}

int or_step(or_sim *S, double dt)
{
    const or_config *c = &S->c;
    const int64_t ncast = 12LL << (2 * c->l_src);
    const int64_t s = S->step;

    /* 1. emission (Sec. 3.1, Eq. 1): new rays march in this same step */
    if (grow_rays(&S->rays, &S->rcap, S->nray + (int64_t)S->ne * ncast)) return -2;
    for (int32_t e = 0; e < S->ne; ++e) {
        double R[9];
        int32_t Rq[9];
        or_rotation(c->seed, e, s, c->rotate, R, Rq);
        double N0 = S->endot[e] * dt / (double)ncast;
        for (int64_t p = 0; p < ncast; ++p) {
            or_ray *r = &S->rays[S->nray++];
            memset(r, 0, sizeof(*r));
            r->l = c->l_src; r->p = p; r->e = e; r->b = (int32_t)s;
            or_direction(c->l_src, p, Rq, r->d);
            for (int b = 0; b < c->nb; ++b) {
                r->N[b] = c->frac[b] * N0;
                S->emitted += r->N[b];
            }
        }
    }

    /* 2-3. march (Sec. 3.1, Eq. 13, 17) and chemistry (Sec. 4.1).  With
     * gamma_iters > 1 the step is repeated from the same start state with the
     * opacity of the time-averaged neutral fraction (and sub-grid opacity) of
     * the previous pass, until the last pass, which is committed. */
    const int iters = c->gamma_iters > 1 ? c->gamma_iters : 1;
    double *yk = c->gen_mode ? S->yion : S->y, *kk = S->kap_sub;
    for (int it = 0; it < iters; ++it) {
        or_ray *out = NULL;
        int64_t nout = 0, ocap = 0;
        or_tally t;
        if (or_march(S, dt, yk, kk, &out, &nout, &ocap, &t)) return -2;
        if (it + 1 < iters) {
            free(out);
            or_chem(S, dt, 0, S->y_est, S->k_est);
            yk = S->y_est;
            kk = S->k_est;
            continue;
        }
        free(S->rays);
        S->rays = out; S->nray = nout; S->rcap = ocap;
        S->absorbed += t.absorbed;
        S->escaped += t.escaped;
        S->near_threshold += t.near;
        if (c->merge && or_merge(S, dt, s, -1)) return -2;
        S->segments_last = t.segs;
        S->segments_total += t.segs;
        S->in_flight = 0.0;
        for (int64_t i = 0; i < S->nray; ++i)
            for (int b = 0; b < c->nb; ++b) S->in_flight += S->rays[i].N[b];
        or_chem(S, dt, 1, NULL, NULL);
    }
    S->step++;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* accessors                                                                  */
/* ------------------------------------------------------------------------- */
void or_get_fields(const or_sim *S, double *gamma, double *xHII, double *T, double *nHI)
{
    for (int64_t i = 0; i < S->ncell; ++i) {
        if (gamma) gamma[i] = S->gamma[i];
        if (xHII) xHII[i] = 1.0 - S->y[i];
        if (T) T[i] = S->T[i];
        if (nHI) nHI[i] = S->nH[i] * S->y[i];
    }
}
void or_get_budget(const or_sim *S, double out[4])
{
    out[0] = S->emitted; out[1] = S->absorbed; out[2] = S->escaped; out[3] = S->in_flight;
}
void or_get_counts(const or_sim *S, int64_t out[5])
{
    out[0] = S->nray; out[1] = S->segments_last; out[2] = S->segments_total;
    out[3] = S->step; out[4] = S->near_threshold;
}
void or_get_segcount(const or_sim *S, int32_t *out)
{
    memcpy(out, S->segcnt, (size_t)S->ncell * sizeof(int32_t));
}
void or_get_deposits(const or_sim *S, double *absd, double *ion)
{
    for (int64_t i = 0; i < S->ncell; ++i) { if (absd) absd[i] = S->absd[i]; if (ion) ion[i] = S->ion[i]; }
}
/* live rays: level, pixel, emitter, birth, direction, photons */
int64_t or_get_rays(const or_sim *S, int32_t *lv, int64_t *pix, int32_t *em, int32_t *birth,
                    int32_t *dir, double *N, int64_t cap)
{
    int64_t n = S->nray < cap ? S->nray : cap;
    for (int64_t i = 0; i < n; ++i) {
        const or_ray *r = &S->rays[i];
        lv[i] = r->l; pix[i] = r->p; em[i] = r->e; birth[i] = r->b;
        for (int a = 0; a < 3; ++a) dir[3 * i + a] = r->d[a];
        for (int b = 0; b < S->c.nb; ++b) N[(int64_t)S->c.nb * i + b] = r->N[b];
    }
    return S->nray;
}
int32_t or_num_emitters(const or_sim *S) { return S->ne; }
int64_t or_config_size(void) { return (int64_t)sizeof(or_config); }

/* Test hook: merge the live rays as at the end of the last step taken
 * (whether or not merging is switched on), with that step's dt; K < 0 takes
 * floor(N_ex * N_RT) from the configuration. */
int or_apply_merge(or_sim *S, double dt, int64_t K)
{
    if (S->step < 1) return -1;
    if (or_merge(S, dt, S->step - 1, K)) return -2;
    S->in_flight = 0.0;
    for (int64_t i = 0; i < S->nray; ++i)
        for (int b = 0; b < S->c.nb; ++b) S->in_flight += S->rays[i].N[b];
    return 0;
}

/* merged-ray fields of the live rays, same order as or_get_rays */
int64_t or_get_rays_aux(const or_sim *S, int32_t *kind, int32_t *vflag, int32_t *A, int64_t *P, double *thr,
                        int64_t cap)
{
    int64_t n = S->nray < cap ? S->nray : cap;
    for (int64_t i = 0; i < n; ++i) {
        const or_ray *r = &S->rays[i];
        kind[i] = r->kind; vflag[i] = r->vflag; A[i] = r->A; thr[i] = r->thr;
        for (int a = 0; a < 3; ++a) P[3 * i + a] = r->P[a];
    }
    return S->nray;
}

/* Test hook: replace the live rays (as they stand after the march of step
 * `step`; the next step taken is step + 1).  Arrays as or_get_rays and
 * or_get_rays_aux return them. */
int or_set_rays(or_sim *S, int64_t step, int64_t n, const int32_t *lv, const int64_t *pix, const int32_t *em,
                const int32_t *birth, const int32_t *dir, const double *N, const int32_t *kind, const int32_t *vflag,
                const int32_t *A, const int64_t *P, const double *thr)
{
    if (grow_rays(&S->rays, &S->rcap, n)) return -1;
    for (int64_t i = 0; i < n; ++i) {
        or_ray *r = &S->rays[i];
        memset(r, 0, sizeof(*r));
        r->l = lv[i]; r->p = pix[i]; r->e = em[i]; r->b = birth[i];
        for (int a = 0; a < 3; ++a) { r->d[a] = dir[3 * i + a]; r->P[a] = P[3 * i + a]; }
        for (int b = 0; b < S->c.nb; ++b) r->N[b] = N[(int64_t)S->c.nb * i + b];
        r->kind = kind[i]; r->vflag = vflag[i]; r->A = A[i]; r->thr = thr[i];
    }
    S->nray = n;
    S->step = step + 1;
    return 0;
}

/* Generalized mode: ionised volume fraction and neutral fraction inside it */
void or_get_gen(const or_sim *S, double *xion, double *yion)
{
    for (int64_t i = 0; i < S->ncell; ++i) {
        if (xion) xion[i] = S->xion[i];
        if (yion) yion[i] = S->yion[i];
    }
}
