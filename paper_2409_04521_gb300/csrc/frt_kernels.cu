// frt_kernels.cu -- the GPU kernels of one RT step and their launchers.
//
//   k_emit   : per active emitter, the step's random sphere rotation and the
//              12*4^l_src new rays at the emitter's cell centre
//              (Sec. 3.1, Eq. 1);
//   k_march  : (frt_march.cuh) per ray, the one-cell march with exp(-tau)
//              attenuation, the Eq. 17 deposit, escape, termination, the
//              Eq. 2-3 split and the compacted write of survivors and children;
//   k_chem   : per cell, Gamma from the deposits, the ionisation update of
//              Sec. 4.1 Eq. 7-10 (double precision), the temperature update
//              of Eq. 12 (single precision) and kappa for the next step;
//   k_end    : per simulation, commit of the step's photon budget.
// All launches are sized on the host from capacities only; counts are read
// from device memory, so the same launches can be replayed in a CUDA graph.
#include <cstdio>
#include "frt_march.cuh"

namespace frt {

// ---------------------------------------------------------------------------
// fixed-point pixel vector table, levels 0..L
// ---------------------------------------------------------------------------
__global__ void k_pixtab(int4 *tab, int L) {
    long long n = level_offset(L + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (level_offset(l + 1) <= i) ++l;
        tab[i] = healpix_vq(l, i - level_offset(l));
    }
}

// ---------------------------------------------------------------------------
// kappa of a cell for the next step (Sec. 4.2, Eq. 13 and the sub-grid law)
// ---------------------------------------------------------------------------
// (single precision throughout; `ionised`: the cell's neutral fraction is at
// most 1 - the ionised threshold of the sub-grid law)
__device__ __forceinline__ float2 cell_kappa(const SimDev &S, float nHf, float yf, bool ionised, float G) {
    const float kx = nHf * yf * S.ksc_f;
    float ks = 0.0f;
    if (S.mfp_mode == 1) {
        ks = S.kap_sub0;
    } else if (S.mfp_mode == 2 && ionised) {
        const float g = fmaxf(G, S.gamma_floor_f);
        const float f = powf(nHf * S.inv_nH_mean_f, S.neg_delta_exp_f) * powf(g * S.inv_gamma_ref_f, S.gamma_exp_f);
        ks = __fdividef(S.kap_sub0, f);
    }
    return make_float2(kx, ks);
}

// Generalized mode (Sec. 4.2): neutral fraction of the highly ionised part
// -- with the photo-ionisation-equilibrium law (mfp mode 3, Eq. 20-22)
// alpha (1 + chi) n_H / Gamma, else 0 -- and its opacity: n_HI sigma from
// that fraction plus the sub-grid law's 1/lambda.  A part never lit yet
// (Gamma = 0) is optically thin (the Eq. 14 guess).
__device__ __forceinline__ float gen_y_ion(const SimDev &S, float nHf, float G, float alpha) {
    if (S.mfp_mode != 3 || !(G > 0.0f)) return 0.0f;
    const float g = fmaxf(G, S.gamma_floor_f);
    return fminf(1.0f, alpha * S.chi1_f * nHf / g);
}
// case-B recombination coefficient of a Generalized-mode cell at T
__device__ __forceinline__ float gen_alpha(const SimDev &S, float T) {
    if (S.isothermal) return S.alpha_iso;
    return S.rates ? alphaB_f(T) : S.alpha_const_f;
}

// Generalized mode with evolving temperature (Sec. 4.2): dT/dt of the
// ionised part from Eq. 12 at static density -- the photo-heating of Eq. 22,
// E_pl alpha_A n_e n_HII (photo-ionisations balance case-A recombinations),
// less the cooling rates with n_HI = y_ion n_H and n_e = n_HII + chi n_H.
// Per n_H^2 inside, pref = 2 n_H / (3 k_B n_tot / n_H).
__device__ __forceinline__ float gen_dTdt_f(const SimDev &S, float T, float yion, float xe, float pref, float cc) {
    const float heat = S.pl_heat * alphaA_f(T) * xe * (1.0f - yion);
    return pref * (heat - cooling_f(T, xe, yion, 1.0f - yion, cc, S.Tcmb));
}
// Newly ionised gas enters at T_reion and mixes by mass with the gas ionised
// before; then sub-steps of the two-stage Rosenbrock scheme ROS2 (Verwer,
// Spee, Blom & Hundsdorfer 1999, gamma = 1 + 1/sqrt 2; second order for any
// Jacobian: here a one-sided difference over 10^-3 T, clipped at 0), each at
// most the step that would move T by 5% explicitly, at most 1000 (the last
// takes what is left).  L-stable: a step much longer than the relaxation
// time ends at the equilibrium temperature.
__device__ float gen_temperature_f(const SimDev &S, float T0, float x0, float dx, float x1, float yion, float nHf) {
    float T = dx > 0.0f ? (x0 * T0 + dx * S.t_reion) / x1 : T0;
    const float xe = 1.0f - yion + S.chi_f;
    const float pref = 2.0f * nHf / (3.0f * KB_F * (S.chi1_f + xe));
    const float cc = S.compton_c / nHf;
    const float gam = 1.70710678f;
    float left = S.dt_f;
    for (int k = 0; k < 1000 && left > 0.0f; ++k) {
        const float f = gen_dTdt_f(S, T, yion, xe, pref, cc);
        if (f == 0.0f) break;
        const float J = fminf((gen_dTdt_f(S, T * 1.001f, yion, xe, pref, cc) - f) / (0.001f * T), 0.0f);
        float h = left;
        if (k < 999) h = fminf(h, 0.05f * T / fabsf(f));
        const float w = 1.0f / (1.0f - gam * h * J);
        const float k1 = w * f;
        const float k2 = w * (gen_dTdt_f(S, T + h * k1, yion, xe, pref, cc) - 2.0f * k1);
        T += h * (1.5f * k1 + 0.5f * k2);
        left -= h;
    }
    return T;
}
__device__ __forceinline__ float2 gen_kappa(const SimDev &S, float nHf, float yion, float G) {
    const float kx = nHf * yion * S.ksc_f;
    float ks = 0.0f;
    if (S.mfp_mode == 1) {
        ks = S.kap_sub0;
    } else if (S.mfp_mode == 2 && G > 0.0f) {
        const float g = fmaxf(G, S.gamma_floor_f);
        const float f = powf(nHf * S.inv_nH_mean_f, S.neg_delta_exp_f) * powf(g * S.inv_gamma_ref_f, S.gamma_exp_f);
        ks = __fdividef(S.kap_sub0, f);
    }
    return make_float2(kx, ks);
}

// e = e^-r, g = (1 - e^-r)/r and h = (1 - g)/r for r >= 0 in single
// precision: Taylor series below r = 1/2, closed forms above.
__device__ __forceinline__ void relax_factors(float r, float &e, float &g, float &h) {
    const float u = fminf(fmaxf(r, 0.0f), 0.5f);
    float sg = 1.0f / 39916800.0f, sh = 1.0f / 479001600.0f;     // 1/11!, 1/12!
    const float cg[10] = {1.0f / 3628800.0f, 1.0f / 362880.0f, 1.0f / 40320.0f, 1.0f / 5040.0f, 1.0f / 720.0f,
                          1.0f / 120.0f, 1.0f / 24.0f, 1.0f / 6.0f, 0.5f, 1.0f};
    const float ch[10] = {1.0f / 39916800.0f, 1.0f / 3628800.0f, 1.0f / 362880.0f, 1.0f / 40320.0f, 1.0f / 5040.0f,
                          1.0f / 720.0f, 1.0f / 120.0f, 1.0f / 24.0f, 1.0f / 6.0f, 0.5f};
#pragma unroll
    for (int k = 0; k < 10; ++k) { sg = fmaf(sg, -u, cg[k]); sh = fmaf(sh, -u, ch[k]); }
    if (r < 0.5f) { g = sg; h = sh; e = 1.0f - r * sg; return; }
    e = __expf(-r);
    g = __fdividef(1.0f - e, r);
    h = __fdividef(1.0f - g, r);
}

__global__ void k_init_cells(const SimDev *sims, int sim, Cells c) {
    const SimDev &S = sims[sim];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.ncell; i += (long long)gridDim.x * blockDim.x) {
        long long g = S.cell_off + i;
        // Generalized mode starts with no ionised fraction
        double y = S.gen_mode ? 1.0 : 1.0 - S.x_init;
        c.y[g] = y;
        c.x[g] = S.gen_mode ? 0.0f : (float)S.x_init;
        c.T[g] = (float)S.T_init;
        c.gamma[g] = 0.0f;
        c.dep[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c.segcnt) c.segcnt[g] = 0;
        c.xion[g] = 0.0;
        c.rho[g] = 1.0f;
        c.fscr[g] = make_float2(0.f, 0.f);
        const float nHf = (float)c.nH[g];
        c.nHf[g] = nHf;
        c.kap[g] = S.gen_mode ? gen_kappa(S, nHf, 0.0f, 0.0f) : cell_kappa(S, nHf, (float)y, y <= S.y_thr, 0.0f);
    }
}

// ---------------------------------------------------------------------------
// emission
// ---------------------------------------------------------------------------
__global__ void k_emit(EmitArgs A) {
    Ctl *C = A.ctl;
    if (C->err) return;
    const int par = C->par;
    const long long base = C->cnt[par];
    const long long total = C->emit_total;
    if (base + total > A.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&C->err, 1);
        return;
    }
    const Queue q = A.q[par];
    const int n = C->n_act_emit;
    const int nr = (n + 31) & ~31;                 // whole warps: the budget sum below is warp-wide
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
        double emitted = 0.0;
        int esim = -1;
        if (j < n) {
        const int e = A.em.act[j];
        const long long off = base + A.em.act_off[j];
        const int4 cell = A.em.cell[e];
        const SimDev &S = A.sims[cell.w];
        const int s = S.step;
        int4 rows[3];
        rotation_rows(S.seed, A.em.local[e], s, S.rotate, rows);
        int4 *ring = A.em.ring + ((long long)e * A.em.ring_w + (s % A.em.ring_w)) * 3;
        ring[0] = rows[0]; ring[1] = rows[1]; ring[2] = rows[2];
        const float n0 = (float)(A.em.ndot[e] * S.dt * S.inv_ncast / S.nref);
        A.em.n0[e] = n0;
        float ph[MAXB];
        double tot = 0.0;
#pragma unroll
        for (int b = 0; b < MAXB; ++b) {
            ph[b] = b < S.nb ? S.frac[b] * n0 : 0.0f;
            tot += (double)ph[b];
        }
        const int l = S.l_src;
        const long long ncast = 12LL << (2 * l);
        const int4 *vt = A.pixtab + level_offset(l <= A.ltab ? l : 0);
        for (long long p = 0; p < ncast; ++p) {
            int32_t dx, dy, dz;
            rotate_dir(rows, l <= A.ltab ? vt[p] : healpix_vq(l, p), dx, dy, dz);
            long long o = off + p;
            q.pl[o] = ((uint32_t)l << LEVEL_SHIFT) | (uint32_t)p;
            q.em[o] = (uint32_t)e;
            q.bi[o] = s;
            q.dx[o] = dx; q.dy[o] = dy; q.dz[o] = dz;
            for (int b = 0; b < A.nb; ++b) q.ph[b][o] = ph[b];
        }
        emitted = tot * (double)ncast;
        esim = cell.w;
        }
        // photons emitted, summed over the warp when its emitters share a
        // simulation (one atomic per warp instead of one per emitter)
        const int kref = __reduce_max_sync(FULL, esim);
        if (kref >= 0) {
            if (__all_sync(FULL, esim < 0 || esim == kref)) {
                double v[1] = {esim == kref ? emitted : 0.0};
                warp_sum<1>(v);
                if (lane_id() == 0) atomicAdd(&A.acc[kref].p_emit, v[0]);
            } else if (esim >= 0) {
                atomicAdd(&A.acc[esim].p_emit, emitted);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// march + deposit + terminate + split + compact
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// chemistry
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_chem(ChemArgs A) {
    // per-simulation absorbed totals and screens' excess photons, then the
    // active cell ranges
    extern __shared__ double sh_abs[];
    double *sh_lost = sh_abs + A.nsims;
    long long *s_pref = reinterpret_cast<long long *>(sh_lost + A.nsims);
    long long *s_cell0 = s_pref + A.nsims + 1;
    int *s_sim = reinterpret_cast<int *>(s_cell0 + A.nsims);
    // Generalized mode: its flag and the atoms of a cell per unit n_H, in
    // code photons
    float *s_apn = reinterpret_cast<float *>(s_sim + A.nsims);
    int *s_gen = reinterpret_cast<int *>(s_apn + A.nsims);
    const Ctl *C = A.ctl;
    const int nrng = C->n_ranges;
    for (int i = threadIdx.x; i < A.nsims; i += blockDim.x) {
        sh_abs[i] = 0.0;
        sh_lost[i] = 0.0;
        const SimDev &S = A.sims[i];
        s_apn[i] = S.apn_f;
        s_gen[i] = S.gen_mode;
    }
    for (int i = threadIdx.x; i <= nrng; i += blockDim.x) s_pref[i] = A.rg.pref[i];
    for (int i = threadIdx.x; i < nrng; i += blockDim.x) { s_cell0[i] = A.rg.cell0[i]; s_sim[i] = A.rg.sim[i]; }
    __syncthreads();
    const bool err = C->err != 0;
    const long long n = C->ncell_active;
    const long long nr = (n + 31) & ~31LL;
    const int lane = lane_id();
    // absorbed photons: each thread sums its cells of one simulation in a
    // register pair (a single-precision sum and its exact rounding error,
    // Knuth's two-sum: no FP64 per cell) and adds the sum to the block's
    // total when the simulation changes and at the end (one shared-memory
    // atomic per run of cells, not one per warp and cell)
    float t_hi = 0.0f, t_lo = 0.0f;
    int t_sim = -1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x) {
        int sim = -1;
        float a_abs = 0.0f;
        if (i < n) {
            int lo = 0, hi = nrng;  // largest r with pref[r] <= i
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (s_pref[mid] <= i) lo = mid; else hi = mid;
            }
            sim = s_sim[lo];
            const long long g = s_cell0[lo] + (i - s_pref[lo]);
            // every load of the cell first: the stores below would otherwise
            // hold the later loads back, one memory round trip each
            const bool gen = s_gen[sim] != 0;
            const float4 d = A.cells.dep[g];
            const float nHf = A.cells.nHf[g];
            const float T0 = A.cells.T[g];
            float2 fs = make_float2(0.f, 0.f);
            double xs;                     // Generalized: x_ion; Standard: neutral fraction y
            float x0f = 0.0f;
            if (gen) {
                fs = A.cells.fscr[g];
                xs = A.cells.xion[g];
            } else {
                xs = A.cells.y[g];
                x0f = A.cells.x[g];
            }
            A.cells.dep[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (A.cells.segcnt) A.cells.segcnt[g] = (int)d.w;
            if (gen) A.cells.fscr[g] = make_float2(0.f, 0.f);
            const SimDev &SG = A.sims[sim];
            if (gen) {
                // Generalized mode (Sec. 4.2): Gamma of the ionised part (Eq. 17
                // with ds -> x ds, V -> x V); the cell's atom balance -- photons
                // absorbed at the screen and in the ionised part less the
                // recombinations there, alpha (1 + chi) n_H^2 x V dt (Eq. 22's
                // approximation) -- moves x (Eq. 18 when the last two cancel);
                // the screen's share rho for the next pass or step
                if (!err) {
                    // single precision except the state x_ion and its
                    // complement (FP64 is a narrow pipe on this part): the
                    // atoms of the cell Ac and the photons in code units, and
                    // the recombinations per atom alpha n_H x dt
                    a_abs = d.x + fs.x;
                    const double x = xs;
                    const float xf = (float)x, omx = (float)(1.0 - x);
                    const float Ac = nHf * s_apn[sim];                           // atoms of a whole cell
                    const float Gf = xf > 0.0f ? d.y * SG.gscale_f / xf : 0.0f;
                    const float alpha = gen_alpha(SG, T0);
                    if (!A.final_pass) {
                        A.cells.rho[g] = fs.y > omx * Ac ? omx * Ac / fs.y : 1.0f;
                        A.cells.kap[g] = gen_kappa(SG, nHf, gen_y_ion(SG, nHf, Gf, alpha), Gf);
                    } else {
                        const float dxf = (fs.x + d.x) / Ac - alpha * nHf * xf * SG.dt_f;
                        const double x1 = fmin(fmax(x + (double)dxf, 0.0), 1.0);
                        // a screen that absorbed more photons than its cell had
                        // neutral atoms (one first reached in the last pass: its
                        // share came from a pass it was not lit in): the excess
                        // ionises nothing
                        const float sx = fs.x - omx * Ac;
                        if (sx > 0.0f) atomicAdd(&sh_lost[sim], (double)sx);
                        const float om1 = (float)(1.0 - x1), x1f = (float)x1;
                        A.cells.rho[g] = fs.y > om1 * Ac ? om1 * Ac / fs.y : 1.0f;
                        // the temperature moves with the start-of-step neutral
                        // fraction; the committed one is that of the new T
                        float yi = gen_y_ion(SG, nHf, Gf, alpha);
                        if (!SG.isothermal && x1 > 0.0) {
                            const float T1 = gen_temperature_f(SG, T0, xf, (float)(x1 - x), x1f, yi, nHf);
                            A.cells.T[g] = T1;
                            yi = gen_y_ion(SG, nHf, Gf, gen_alpha(SG, T1));
                        }
                        A.cells.xion[g] = x1;
                        A.cells.y[g] = fma(x1, (double)yi, 1.0 - x1);
                        A.cells.x[g] = x1f * (1.0f - yi);
                        A.cells.gamma[g] = Gf;
                        A.cells.kap[g] = gen_kappa(SG, nHf, yi, Gf);
                    }
                }
            } else if (!err) {
                a_abs = d.x;
                const SimDev &S = A.sims[sim];
                const float Gf = d.y * S.gscale_f;                    // Eq. 17, 1/s
                const double y0 = xs;
                const float y0f = (float)y0;
                const float dtf = S.dt_f;
                float alpha = S.alpha_iso, Cc = S.coll_iso;
                if (!S.isothermal && S.rates) { alpha = alphaB_f(T0); Cc = collion_f(T0); }
                else if (!S.isothermal) alpha = S.alpha_const_f;
                // Eq. 7-10 with n_e re-evaluated from <x>.  With i = Gamma + C n_e,
                // b = alpha n_e, r = dt (i + b), e = e^-r, g = (1 - e)/r and
                // h = (1 - g)/r, the solution x(t) = x_eq + (x0 - x_eq) e^{-t/t_i}
                // and its time average are, for y = 1 - x,
                //   x1 = x0 e + g i dt,  y1 = y0 e + g b dt,
                //   <x> = x0 g + h i dt, <y> = y0 g + h b dt:
                // sums of positive terms, accurate however small x or y is.
                float xb = x0f, yb = y0f, ef = 1.0f, gf = 0.0f, hf = 0.0f, idt = 0.0f, bdt = 0.0f;
                for (int it = 0; it < S.chem_iters; ++it) {
                    const float ne = nHf * xb;
                    idt = (Gf + Cc * ne) * dtf;
                    bdt = alpha * ne * dtf;
                    relax_factors(idt + bdt, ef, gf, hf);
                    const float xbn = fmaf(x0f, gf, hf * idt);
                    yb = fmaf(y0f, gf, hf * bdt);
                    const bool conv = fabsf(xbn - xb) <= 1e-7f * xbn;
                    xb = xbn;
                    if (conv) break;
                }
                if (!A.final_pass) {
                    // a trial pass of the Gamma - <n_HI> iteration (Eq. 11; with
                    // the sub-grid law lambda - Gamma): the next march sees the
                    // opacity of the time-averaged state; the state is kept
                    A.cells.kap[g] = cell_kappa(S, nHf, yb, yb <= S.y_thr_dn, Gf);
                } else {
                // x1 + y1 = 1 holds to rounding: keep x1 in [0, 1]
                const float x1 = fminf(fmaf(x0f, ef, gf * idt), 1.0f);
                const double y1 = fma(y0, (double)ef, (double)(gf * bdt));   // neutral fraction kept in FP64
                float T = T0;
                if (!S.isothermal) {
                    // Eq. 12 with static density: particle-number term, then
                    // sub-stepped heating minus cooling (per n_H^2)
                    T = T0 * (1.0f + x0f) / (1.0f + x1);
                    const float heat = d.z * S.hscale_f * yb / nHf;
                    const float pref = 2.0f * nHf / (3.0f * KB_F * (1.0f + xb));
                    const float cc = S.compton_c / nHf;
                    float left = dtf;
                    for (int k = 0; k < 1000 && left > 0.0f; ++k) {
                        const float lam = cooling_f(T, xb, yb, xb, cc, S.Tcmb);
                        const float dTdt = pref * (heat - lam);
                        float h = left;
                        if (k < 999 && dTdt != 0.0f) h = fminf(h, 0.05f * T / fabsf(dTdt));
                        T += dTdt * h;
                        left -= h;
                    }
                }
                A.cells.y[g] = y1;
                A.cells.x[g] = x1;
                A.cells.T[g] = T;
                A.cells.gamma[g] = Gf;
                A.cells.kap[g] = cell_kappa(S, nHf, (float)y1, y1 <= S.y_thr, Gf);
                }
            }
        }
        if (sim >= 0 && a_abs != 0.0f) {
            if (sim != t_sim) {
                if (t_sim >= 0) atomicAdd(&sh_abs[t_sim], (double)t_hi + (double)t_lo);
                t_sim = sim;
                t_hi = t_lo = 0.0f;
            }
            const float s = t_hi + a_abs, bp = s - t_hi;
            t_lo += (t_hi - (s - bp)) + (a_abs - bp);
            t_hi = s;
        }
    }
    {
        // the warp's sums: one atomic when its lanes share a simulation
        const double t_abs = (double)t_hi + (double)t_lo;
        const int kref = __reduce_max_sync(FULL, t_sim);
        if (kref >= 0 && __all_sync(FULL, t_sim < 0 || t_sim == kref)) {
            double v[1] = {t_sim == kref ? t_abs : 0.0};
            warp_sum<1>(v);
            if (lane == 0 && v[0] != 0.0) atomicAdd(&sh_abs[kref], v[0]);
        } else if (t_sim >= 0 && t_abs != 0.0) {
            atomicAdd(&sh_abs[t_sim], t_abs);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < A.nsims; i += blockDim.x) {
        if (sh_abs[i] != 0.0) atomicAdd(&A.acc[i].p_abs, sh_abs[i]);
        if (sh_lost[i] != 0.0) atomicAdd(&A.acc[i].p_lost, sh_lost[i]);
    }
}

// ---------------------------------------------------------------------------
// end of step
// ---------------------------------------------------------------------------
__global__ void k_end(Ctl *C, SimDev *sims, SimAcc *acc, int nsims) {
    const bool err = C->err != 0;
    for (int j = threadIdx.x; j < nsims; j += blockDim.x) {
        SimAcc &a = acc[j];
        if (!err && sims[j].active) {
            a.emitted += a.p_emit;
            a.absorbed += a.p_abs;
            a.escaped += a.p_esc;
            a.in_flight = a.p_out;
            a.seg_last = a.p_seg;
            a.seg_total += a.p_seg;
            a.rays_live = a.p_rays_out;
            a.rays_in_last = a.p_rays_in;
            a.rays_in_total += a.p_rays_in;
            a.lost += a.p_lost;
            sims[j].step += 1;
        }
        a.p_emit = a.p_abs = a.p_esc = a.p_out = a.p_in = 0.0;
        a.p_seg = a.p_rays_in = a.p_rays_out = a.p_lost = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the march wrote the live rays to the other queue (a merge step
        // left holes there, which the next march skips)
        const int par = C->par;
        if (err) C->cnt[par ^ 1] = 0;
        else {
            C->cnt[par] = 0;
            C->par = par ^ 1;
        }
        C->merged = 0;
    }
}

// between passes of the Gamma - <n_HI> iteration: the next pass marches the
// same rays again, so the march's output and the step's tallies are dropped
// (emission happens once per step; the marched-ray counter keeps every pass)
__global__ void k_iter_reset(Ctl *C, SimAcc *acc, int nsims) {
    if (C->err) return;
    for (int j = threadIdx.x; j < nsims; j += blockDim.x) {
        SimAcc &a = acc[j];
        a.rays_in_total += a.p_rays_in;
        a.p_abs = a.p_esc = a.p_out = a.p_in = 0.0;
        a.p_seg = a.p_rays_in = a.p_rays_out = a.p_lost = 0.0;
    }
    if (threadIdx.x == 0) C->cnt[C->par ^ 1] = 0;
}

// ---------------------------------------------------------------------------
// probes: the same device functions on host-given inputs
// ---------------------------------------------------------------------------
__global__ void k_probe_pixvec(int level, long long p0, long long n, int32_t *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int4 v = healpix_vq(level, p0 + i);
        out[3 * i] = v.x; out[3 * i + 1] = v.y; out[3 * i + 2] = v.z;
    }
}
// the single-precision rate fits of the chemistry kernel (Sec. 4.1) at n
// temperatures: alpha_B, alpha_A, C_HI and the cooling rate with unit
// electron, HI and HII fractions and no Compton term
__global__ void k_probe_rates(long long n, const float *T, float *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float t = T[i];
        out[4 * i + 0] = alphaB_f(t);
        out[4 * i + 1] = alphaA_f(t);
        out[4 * i + 2] = collion_f(t);
        out[4 * i + 3] = cooling_f(t, 1.0f, 1.0f, 1.0f, 0.0f, 0.0f);
    }
}
__global__ void k_probe_rotation(uint64_t seed, long long e, long long s, int rotate, int32_t *out) {
    int4 r[3];
    rotation_rows(seed, e, s, rotate, r);
    for (int k = 0; k < 3; ++k) { out[3 * k] = r[k].x; out[3 * k + 1] = r[k].y; out[3 * k + 2] = r[k].z; }
}
__global__ void k_probe_direction(int level, long long p0, long long n, const int32_t *Rq, const int4 *tab, int ltab,
                                  int32_t *out) {
    int4 rows[3];
    for (int k = 0; k < 3; ++k) rows[k] = make_int4(Rq[3 * k], Rq[3 * k + 1], Rq[3 * k + 2], 0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long p = p0 + i;
        int4 v = level <= ltab ? tab[level_offset(level) + p] : healpix_vq(level, p);
        int32_t dx, dy, dz;
        rotate_dir(rows, v, dx, dy, dz);
        out[3 * i] = dx; out[3 * i + 1] = dy; out[3 * i + 2] = dz;
    }
}
__global__ void k_probe_traverse(long long n, const long long *p0, const int32_t *d, int gx, int gy, int gz,
                                 int32_t *cells, float *ds, int32_t *nseg, int32_t *esc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        Walk w;
        walk_init(w, (int)p0[3 * i], (int)p0[3 * i + 1], (int)p0[3 * i + 2], d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        int key[4];
        float s[4];
        bool e = false;
        const unsigned m = walk_step(w, gx, gy, gz, 0, key, s, e);
        int k = 0;
        for (int j = 0; j < 4; ++j) {
            if (!(m & (1u << j))) continue;
            const int c = key[j];
            cells[12 * i + 3 * k] = c % gx;
            cells[12 * i + 3 * k + 1] = (c / gx) % gy;
            cells[12 * i + 3 * k + 2] = c / (gx * gy);
            ds[4 * i + k] = s[j];
            ++k;
        }
        nseg[i] = k;
        esc[i] = e ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pixtab(int4 *tab, int L, cudaStream_t st) {
    long long n = level_offset(L + 1);
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    k_pixtab<<<blocks, 256, 0, st>>>(tab, L);
    return cudaGetLastError();
}
cudaError_t launch_init_cells(const SimDev *sims, int sim, Cells c, long long ncell, cudaStream_t st) {
    int blocks = (int)((ncell + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_init_cells<<<blocks, 256, 0, st>>>(sims, sim, c);
    return cudaGetLastError();
}
cudaError_t launch_emit(const EmitArgs &a, int blocks, cudaStream_t st) {
    k_emit<<<blocks, 128, 0, st>>>(a);
    return cudaGetLastError();
}
// Kernel variants: every bin count with the default (AGG 0, 2 blocks/SM);
// the bin counts of the standard spectra (1, 3, 4) with every aggregation
// and register budget, for the autotuner.  The variants with merged rays
// are built in frt_merge.cu, those that also run Generalized members in
// frt_march_gen.cu.
static MarchFn march_fn_plain(int nb, int agg, int minb) {
#define FRT_V(NB)                                                                   \
    if (nb == NB) {                                                                \
        if (agg == 0 && minb == 2) return k_march<NB, 0, 2, 0>;                    \
        if (agg == 0 && minb == 3) return k_march<NB, 0, 3, 0>;                    \
        if (agg == 0 && minb == 4) return k_march<NB, 0, 4, 0>;                    \
        if (agg == 1 && minb == 2) return k_march<NB, 1, 2, 0>;                    \
        if (agg == 1 && minb == 3) return k_march<NB, 1, 3, 0>;                    \
        if (agg == 1 && minb == 4) return k_march<NB, 1, 4, 0>;                    \
        if (agg == 2 && minb == 2) return k_march<NB, 2, 2, 0>;                    \
        if (agg == 2 && minb == 3) return k_march<NB, 2, 3, 0>;                    \
        if (agg == 2 && minb == 4) return k_march<NB, 2, 4, 0>;                    \
        return nullptr;                                                            \
    }
    FRT_V(1)
    FRT_V(3)
    FRT_V(4)
#undef FRT_V
    if (agg != 0 || minb != 2) return nullptr;
    switch (nb) {
        case 2: return k_march<2, 0, 2, 0>;
        case 5: return k_march<5, 0, 2, 0>;
        case 6: return k_march<6, 0, 2, 0>;
        case 7: return k_march<7, 0, 2, 0>;
        case 8: return k_march<8, 0, 2, 0>;
        default: return nullptr;
    }
}
static MarchFn march_fn(int nb, int agg, int minb, int ext) {
    switch (ext) {
        case 0: return march_fn_plain(nb, agg, minb);
        case 1: return march_fn_merge(nb, agg, minb);
        case 3: return march_fn_gen(nb, agg, minb);
        default: return nullptr;
    }
}
bool march_variant_exists(int nb, int agg, int minb, int ext) { return march_fn(nb, agg, minb, ext) != nullptr; }
cudaError_t march_prepare(int nb, int agg, int minb, int nsims, int ext) {
    MarchFn f = march_fn(nb, agg, minb, ext);
    if (!f) return cudaErrorInvalidValue;
    const size_t sh = march_shared_bytes(nsims);
    if (sh > 48 * 1024) return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    return cudaSuccess;
}
cudaError_t launch_march(const MarchArgs &a, int nb, int agg, int minb, int blocks, int threads, cudaStream_t st,
                         int ext) {
    MarchFn f = march_fn(nb, agg, minb, ext);
    if (!f) return cudaErrorInvalidValue;
    f<<<blocks, threads, march_shared_bytes(a.nsims), st>>>(a);
    return cudaGetLastError();
}
int march_max_blocks_per_sm(int nb, int agg, int minb, int threads, int nsims, int ext) {
    MarchFn f = march_fn(nb, agg, minb, ext);
    if (!f) return 0;
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, march_shared_bytes(nsims));
    return n;
}
cudaError_t launch_chem(const ChemArgs &a, int blocks, cudaStream_t st) {
    const size_t sh = (size_t)a.nsims * 2 * sizeof(double) + (size_t)(2 * a.nsims + 1) * sizeof(long long) +
                      (size_t)a.nsims * (2 * sizeof(int) + sizeof(float));
    k_chem<<<blocks, 256, sh, st>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_iter_reset(Ctl *c, SimAcc *acc, int nsims, cudaStream_t st) {
    k_iter_reset<<<1, 256, 0, st>>>(c, acc, nsims);
    return cudaGetLastError();
}
cudaError_t launch_end(Ctl *c, SimDev *sims, SimAcc *acc, int nsims, cudaStream_t st) {
    k_end<<<1, 256, 0, st>>>(c, sims, acc, nsims);
    return cudaGetLastError();
}
cudaError_t launch_probe_pixvec(int level, long long p0, long long n, int32_t *out, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_probe_pixvec<<<blocks, 256, 0, st>>>(level, p0, n, out);
    return cudaGetLastError();
}
cudaError_t launch_probe_rates(long long n, const float *T, float *out, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    k_probe_rates<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(n, T, out);
    return cudaGetLastError();
}
cudaError_t launch_probe_rotation(uint64_t seed, long long e, long long s, int rotate, int32_t *out, cudaStream_t st) {
    k_probe_rotation<<<1, 1, 0, st>>>(seed, e, s, rotate, out);
    return cudaGetLastError();
}
cudaError_t launch_probe_direction(int level, long long p0, long long n, const int32_t *Rq, const int4 *tab, int ltab,
                                   int32_t *out, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_probe_direction<<<blocks, 256, 0, st>>>(level, p0, n, Rq, tab, ltab, out);
    return cudaGetLastError();
}
cudaError_t launch_probe_traverse(long long n, const long long *p0, const int32_t *d, int gx, int gy, int gz,
                                  int32_t *cells, float *ds, int32_t *nseg, int32_t *esc, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_probe_traverse<<<blocks, 256, 0, st>>>(n, p0, d, gx, gy, gz, cells, ds, nseg, esc);
    return cudaGetLastError();
}

}  // namespace frt
