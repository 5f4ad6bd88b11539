// frt_types.h -- data layout shared by the step kernels and the host engine.
//
// Units on the device ("code units"): lengths in cells, one step moves a ray
// one cell (Sec. 3.1), positions and directions in 2^-21 cell fixed point,
// photons in units of a per-simulation reference count nref, opacities as
// optical depth per cell at the reference cross-section sigma_ref.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace frt {

constexpr int FRAC_BITS = 21;                       // position fixed point
constexpr int64_t ONE_CELL = int64_t(1) << FRAC_BITS;
constexpr int VQ_BITS = 24;                         // pixel vectors / rotations
constexpr int MAXB = 8;                             // frequency bins
constexpr int MAXL = 13;                            // HEALPix levels 0..12
constexpr int LEVEL_SHIFT = 28;                     // pixlev = level<<28 | pixel
constexpr uint32_t PIX_MASK = (1u << LEVEL_SHIFT) - 1u;
constexpr uint32_t DEAD_RAY = 0xffffffffu;         // unused queue slot (level 15 never occurs)
constexpr int OUT_SLAB = 512;                       // queue slots a warp reserves at once
constexpr uint32_t MERGED_BIT = 0x80000000u;        // emitter word of a merged ray: bit | local cell
constexpr int HIST_BINS = 65536;                    // radix-select bins per pass (16 bits)
constexpr int MERGE_MAX_BLOCKS = 4096;              // blocks of the merge's per-ray passes (8 warps each)

// Per-simulation constants and step state.
struct SimDev {
    int32_t nx, ny, nz, nb;
    int64_t cell_off, ncell;
    int32_t l_src, l_max;
    int32_t K[16];          // split after (age+1) >= K[l] whole steps (Eq. 2)
    int32_t active;         // takes part in steps
    int32_t step;           // steps taken
    int32_t ring_w;         // rotation ring length (> largest ray age)
    int32_t rotate;
    uint64_t seed;
    float eps_term;
    float sig[MAXB];        // sigma_b / sigma_ref
    float sige[MAXB];       // sigma_b / sigma_ref * eheat_b / 1 eV
    float eh[MAXB];         // eheat_b / 1 eV
    float frac[MAXB];       // photon fraction per bin
    double dt;              // s
    double gscale;          // Gamma per unit of the Gamma numerator: nref sigma_ref / (dx^2 dt)
    double hscale;          // heating (erg/s per HI atom) per unit of the heating numerator
    double ksc;             // sigma_ref * dx_phys: tau per cell per (n_HI in cm^-3)
    double inv_nH_mean, inv_gamma_ref, y_thr;  // 1/<n_H>, 1/Gamma_ref, 1 - x threshold
    float kap_sub0;         // dx_com / lambda0
    float alpha_iso, coll_iso;  // rate coefficients at T_init (isothermal runs)
    float compton_c;        // Compton cooling coefficient at this redshift (erg s^-1 K^-1)
    float Tcmb;             // K
    double nref;            // photons per code photon
    double sigma_ref;       // cm^2
    double dx_phys;         // cm
    double dx_com;          // cm comoving
    double inv_ncast;       // 1 / (12 * 4^l_src)
    double z;
    double alpha_const;
    int32_t rates, isothermal, chem_iters, mfp_mode;
    double lambda0_c, delta_exp, gamma_ref, gamma_exp, gamma_floor, xion_thr, nH_mean;
    double x_init, T_init;
    // ray merging (Sec. 3.3): on/off, merge-sphere level, directions, and the
    // number of rays exempt from merging, floor(N_ex * N_RT)
    int32_t merge, l_merge, ndir, pad_m;
    long long k_ex;
    int32_t gamma_iters;    // passes of the Gamma - <n_HI> iteration per step (Sec. 4.1, Eq. 11)
    int32_t gen_mode;       // Generalized Opacity mode (Sec. 4.2): ionised fraction + moving screen
    double chi;             // He/H number ratio (Eq. 18)
    // Generalized mode with evolving temperature: T of newly ionised gas (K)
    // and the Eq. 22 mean excess energy per photo-ionisation (erg)
    float t_reion, pl_heat;
    // single-precision copies for the per-cell chemistry (converting the
    // double fields above in every cell kept the narrow FP64 pipe busy)
    float dt_f, gscale_f, hscale_f, pad_f;       // with dt
    float ksc_f, inv_nH_mean_f, inv_gamma_ref_f, neg_delta_exp_f, gamma_exp_f, gamma_floor_f;
    float y_thr_dn;                              // largest float <= y_thr (same decisions for float y)
    float alpha_const_f, chi_f, chi1_f;          // alpha_const, chi, 1 + chi
    float apn_f;                                 // (1 + chi) V / nref: atoms of a cell per unit n_H
};

// Per-simulation accumulators, code photons (double) and counters.
struct SimAcc {
    double emitted, absorbed, escaped, in_flight;     // committed
    double p_emit, p_abs, p_esc, p_out, p_in;         // current step
    double p_seg, p_rays_in, p_rays_out;              // current step
    double seg_last, seg_total, rays_live, rays_in_last;
    // Generalized mode: photons a screen absorbed beyond the atoms it had
    // (ionising nothing), this step and committed
    double p_lost, lost;
    double rays_in_total;   // marched rays since creation (kept by a reset: last)
};

// Global control words of one engine.
struct Ctl {
    long long cnt[2];        // rays in queue 0 / 1
    int32_t par;             // queue holding the live rays
    int32_t err;             // latched error (bit 0 capacity, bit 1 age, bit 2 level)
    long long emit_total;    // rays emitted per step by the active emitters
    int32_t n_act_emit;      // active emitters
    int32_t n_ranges;        // active cell ranges
    long long ncell_active;  // cells in active simulations
    int32_t merged;          // a simulation merged rays this step
    int32_t pad;
    long long mbase;         // the march's output count: merged rays are appended from here
    long long pad2;
};

// Structure-of-arrays ray queue.
struct Queue {
    uint32_t *pl;            // level << 28 | NESTED pixel
    uint32_t *em;            // emitter id
    int32_t *bi;             // birth step
    int32_t *dx, *dy, *dz;   // direction, 2^-21 cell per step
    float *ph[MAXB];         // code photons per bin
    // merged rays only (Sec. 3.3); null when merging is not built in
    int32_t *mx, *my, *mz;   // position at the merge, 2^-21 cell
    uint32_t *ma;            // vertex << 31 | simulation << 16 | distance travelled at the merge
    float *mthr;             // termination threshold, code photons
};

struct Cells {
    double *nH;              // cm^-3 physical
    float *nHf;              // the same in single precision (chemistry)
    double *y;               // neutral fraction x_HI
    float *x;                // ionised fraction x_HII (kept separately: accurate when small)
    float *T;                // K
    float *gamma;            // Gamma_HI of the last step, 1/s
    float2 *kap;             // (tau per cell at sigma_ref from HI, sub-grid tau per cell)
    float4 *dep;             // (absorbed, Gamma numerator, heating numerator, segments)
    int32_t *segcnt;         // segments of the last step (diagnostics) or null
    // Generalized Opacity mode (Sec. 4.2)
    double *xion;            // highly ionised volume fraction (double: it takes per-step
                             // residuals far below float resolution near 1)
    float *rho;              // share of the photons reaching the screen that it absorbs
    float2 *fscr;            // this pass: photons the screen absorbed, photons that reached it
};

struct Emitters {
    int4 *cell;              // (i, j, k, sim)
    int32_t *local;          // index within its simulation (rotation key)
    double *ndot;            // photons / s
    float *n0;               // this step's code photons per emitted ray
    int4 *ring;              // [emitter][ring slot][3] rotation rows (2^24)
    int32_t ring_w;          // slots per emitter (same for all)
    int32_t *act;            // active emitter ids
    long long *act_off;      // first emitted ray of each active emitter
};

// Scratch of the merge step (Sec. 3.3).
struct MergeWork {
    uint32_t *hist;          // [slot][hrep][HIST_BINS] radix-select counts
    uint32_t *sel;           // [slot][8]: selection state, upper bits, rays above, T_ref bits, any exempt
    uint32_t *tkey;          // per queue slot: rank content (float bits)
    int32_t *tsim;           // per queue slot: simulation taking part, -1 none
    float *grp;              // [cell * ndir + pixel][grp_w]: 6 uint64 weighted sums, photons, threshold
    uint4 *gcm;              // [cell * ndir + pixel] group size, largest member content (float
                             // bits), complement of the lowest candidate-list index (its
                             // leader), unused; all zero when the group is empty
    uint32_t *cand;          // candidate lists, one run per block of the merge passes: the queue
                             // slot of each ray that may merge
    uint32_t *ckey;          // and its rank content (float bits)
    uint4 *tgrp;             // per candidate: group slot (0xffffffff: none), then the end point's
                             // offsets in its cell, distance travelled and level, packed
    int4 *rot;               // [cell][3] merge-sphere rotation rows of this step
    uint32_t *lead_slot;     // merged-ray lists, one run per block: the group slot
    int32_t *lead_sim;       // and the simulation of each merged ray
    uint32_t *bcnt;          // per block of the merge passes: candidates listed
    uint32_t *bled;          // and merged rays listed
    long long lead_cap;      // entries of the candidate and merged-ray lists
    int32_t ndir;            // group slots per cell (12 * 4^l_merge of the deepest allowed level)
    int32_t grp_w;           // floats per group
    int32_t hrep;            // copies of each simulation's histogram (spreads hot bins)
    int32_t pad;
};

struct Ranges {              // active cell ranges for the chemistry kernel
    long long *pref;         // prefix of range sizes [n+1]
    long long *cell0;        // first global cell
    int32_t *sim;            // owning simulation
};

}  // namespace frt
