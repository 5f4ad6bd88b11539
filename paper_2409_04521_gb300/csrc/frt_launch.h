// frt_launch.h -- kernel argument blocks and launchers (host side).
#pragma once
#include <string>
#include "frt_types.h"

namespace frt {

struct EmitArgs {
    Ctl *ctl;
    const SimDev *sims;
    SimAcc *acc;
    Queue q[2];
    long long cap;
    Emitters em;
    const int4 *pixtab;
    int ltab;
    int nb;
};

struct MarchArgs {
    Ctl *ctl;
    const SimDev *sims;
    SimAcc *acc;
    int nsims;
    Queue q[2];
    long long cap;
    Emitters em;
    Cells cells;
    const int4 *pixtab;
    int ltab;
    int slab;                // output slots a warp reserves at once (run length, 32..4096)
};

struct MergeArgs {
    Ctl *ctl;
    const SimDev *sims;
    SimAcc *acc;
    int nsims;
    Queue q[2];
    Emitters em;
    Ranges rg;
    const int4 *pixtab;
    int ltab;
    MergeWork w;
    int nbq;                 // photon bins of the queue layout
    long long cap;           // queue slots (merged rays are appended)
};

struct ChemArgs {
    const Ctl *ctl;
    const SimDev *sims;
    SimAcc *acc;
    int nsims;
    Cells cells;
    Ranges rg;
    int final_pass;          // 0: a trial pass of the Gamma - <n_HI> iteration (state unchanged)
};

// message of the last failed call that has no context (this host thread)
void set_free_error(const std::string &msg);

cudaError_t launch_pixtab(int4 *tab, int L, cudaStream_t st);
cudaError_t launch_init_cells(const SimDev *sims, int sim, Cells c, long long ncell, cudaStream_t st);
cudaError_t launch_emit(const EmitArgs &a, int blocks, cudaStream_t st);
using MarchFn = void (*)(MarchArgs);
// the march variant with merged rays (nullptr if not built)
MarchFn march_fn_merge(int nb, int agg, int minb);
// the variant with merged rays and Generalized Opacity mode (nullptr if not built)
MarchFn march_fn_gen(int nb, int agg, int minb);
// ext: 0 plain, 1 merged rays, 3 merged rays and Generalized mode
bool march_variant_exists(int nb, int agg, int minb, int ext);
// opt the variant into the dynamic shared memory `nsims` slots need
cudaError_t march_prepare(int nb, int agg, int minb, int nsims, int ext);
cudaError_t launch_march(const MarchArgs &a, int nb, int agg, int minb, int blocks, int threads, cudaStream_t st,
                         int ext);
int march_max_blocks_per_sm(int nb, int agg, int minb, int threads, int nsims, int ext);
cudaError_t launch_chem(const ChemArgs &a, int blocks, cudaStream_t st);
cudaError_t launch_end(Ctl *c, SimDev *sims, SimAcc *acc, int nsims, cudaStream_t st);
// between passes of the iteration: drop the march's output and the step's tallies (not emission)
cudaError_t launch_iter_reset(Ctl *c, SimAcc *acc, int nsims, cudaStream_t st);
// the merge step (Sec. 3.3) between the march and the chemistry
// a second stream for the merge's independent rotation pass, with the events
// that fork it from the step's stream and join it back
struct MergeSide {
    cudaStream_t st;
    cudaEvent_t fork, join;
};
cudaError_t launch_merge(const MergeArgs &a, int sm_count, cudaStream_t st, const MergeSide *side);
cudaError_t launch_probe_merge_pixel(int level, long long n, const int32_t *d, const int32_t *Rq, bool per_ray,
                                     uint32_t *out, cudaStream_t st);
cudaError_t launch_probe_pixvec(int level, long long p0, long long n, int32_t *out, cudaStream_t st);
cudaError_t launch_probe_rates(long long n, const float *T, float *out, cudaStream_t st);
cudaError_t launch_probe_rotation(uint64_t seed, long long e, long long s, int rotate, int32_t *out, cudaStream_t st);
cudaError_t launch_probe_direction(int level, long long p0, long long n, const int32_t *Rq, const int4 *tab, int ltab,
                                   int32_t *out, cudaStream_t st);
cudaError_t launch_probe_traverse(long long n, const long long *p0, const int32_t *d, int gx, int gy, int gz,
                                  int32_t *cells, float *ds, int32_t *nseg, int32_t *esc, cudaStream_t st);

}  // namespace frt
