// frt_engine.h -- host engine shared by the single-simulation context and
// the batch: device arenas for cells, emitters and the ray queues, slots of
// simulations, launch configuration, optional CUDA-graph replay of a step.
#pragma once
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/flexrt.h"
#include "frt_launch.h"

namespace frt {

// Process-wide fixed-point pixel-vector table of levels 0..level on `device`.
cudaError_t get_pixtab(int device, int level, cudaStream_t st, const int4 **out);

// First-fit allocator of [0, capacity) index ranges.
class RangeAllocator {
  public:
    void reset(long long capacity);
    long long alloc(long long n);          // -1 if no room
    void release(long long start, long long n);
    long long capacity() const { return cap_; }
    long long used() const { return used_; }

  private:
    struct Free { long long start, n; };
    std::vector<Free> free_;
    long long cap_ = 0, used_ = 0;
};

struct Slot {
    bool used = false;         // holds a simulation (active or retiring)
    bool active = false;       // takes part in steps
    SimDev h{};                // host copy of the constants
    long long cell0 = 0;
    std::vector<int4> ecell;   // per emitter of this simulation (x, y, z, slot)
    std::vector<double> endot;
    long long em0 = -1;        // first global emitter id of the slot's range
    int em_n = 0;              // emitters in the range
    bool nref_set = false;
    int release_after = -1;    // engine step after which the emitter range is freed
};

struct EngineConfig {
    int nb = 1;                // frequency bins of the queue layout
    int max_sims = 1;
    long long ray_capacity = 0;
    long long cell_capacity = 0;
    int emitter_capacity = 0;  // 0 = grow on demand (single simulation only)
    int max_grid = 0;          // largest grid edge (rotation ring length)
    int l_max = FLEXRT_MAX_LEVEL;
    double n_ray_min = 3.0;
    bool keep_diagnostics = false;
    bool use_graph = false;
    void *stream = nullptr;
    int merge_l_max = -1;      // deepest merge-sphere level members may use; -1: no merging
    bool gen_capable = false;  // members may run Generalized Opacity mode
    long long device_bytes_max = 0;  // cap on the engine's device allocations (0 = none)
};

class Engine {
  public:
    ~Engine();
    flexrt_status init(const EngineConfig &cfg);
    // Fill a simulation's constants from the public parameters (no device work).
    static flexrt_status make_sim(const flexrt_grid *grid, const flexrt_box *box, const double *n_H,
                                  const flexrt_mfp *mfp, const flexrt_spectrum *sp, const flexrt_options *opt,
                                  SimDev &h, std::string &err);
    flexrt_status add_sim(const SimDev &h, const double *n_H, int *slot);
    flexrt_status add_sources(int slot, int32_t n, const int32_t *ijk, const double *ndot);
    flexrt_status set_dt(int slot, double dt);
    flexrt_status step();                     // one RT step of every active simulation
    // a single simulation's step in two stages: 1 = emission and marches,
    // 2 = merge, chemistry, commit (the rays getters read the march's output
    // in between)
    flexrt_status step_stage(int stage);
    flexrt_status sync();
    flexrt_status retire(int slot);
    flexrt_status reset_all();                // single-simulation reset
    flexrt_status fields(int slot, flexrt_fields *f);
    flexrt_status budget(int slot, double out[4]);
    flexrt_status screen_excess(int slot, double *out);   // Generalized mode: photons absorbed beyond the atoms
    flexrt_status counts(int slot, int64_t out[6]);
    flexrt_status segment_counts(int slot, int32_t *out);
    flexrt_status rays(int slot, int64_t cap, int32_t *level, int64_t *pixel, int32_t *emitter, int32_t *birth,
                       int32_t *dir, double *photons, int64_t *n);
    flexrt_status rays_merged(int slot, int64_t cap, int32_t *merged, int32_t *vertex, int32_t *dist, int64_t *pos,
                              double *thr, int64_t *n);
    bool merge_built() const { return cfg_.merge_l_max >= 0; }
    // the march variants: 0 plain, 1 with merged rays, 3 with merged rays
    // and the moving screen (engines that may run Generalized members)
    int ext_variants() const { return cfg_.gen_capable ? 3 : (merge_built() ? 1 : 0); }
    flexrt_status ionized_volume(int slot, double *x_ion);
    // checkpoint of a single-simulation engine (slot 0): bytes needed, save, load
    flexrt_status save_state(int slot, void *buf, int64_t cap, int64_t *bytes);
    flexrt_status load_state(int slot, const void *buf, int64_t bytes);
    long long device_bytes() const { return alloc_bytes_; }
    flexrt_status set_launch(int agg, int minb, int blocks_per_sm, int threads, int slab);
    flexrt_status profile(bool on);
    flexrt_status kernel_times(double ms[4], int64_t launches[4], int64_t *rays);
    int active_count() const;
    int free_slots() const;
    flexrt_status queue_used(long long *n);   // queue slots after the last step seen complete
    long long cells_free() const { return cell_alloc_.capacity() - cell_alloc_.used(); }
    long long emitters_free() const { return em_alloc_.capacity() - em_alloc_.used(); }
    const Slot *slot(int s) const { return (s >= 0 && s < (int)slots_.size() && slots_[s].used) ? &slots_[s] : nullptr; }
    int nb() const { return cfg_.nb; }
    long long ray_capacity() const { return cfg_.ray_capacity; }
    const std::string &error() const { return err_; }
    flexrt_status fail(flexrt_status s, const std::string &m) { err_ = m; return s; }
    flexrt_status cuda(cudaError_t e, const char *what);

  private:
    cudaError_t dev_alloc(void **p, size_t bytes);
    void dev_free(void *p);
    flexrt_status grow_emitters(int need);
    flexrt_status upload_lists();             // active emitters, cell ranges, counters
    flexrt_status poll(bool wait);
    flexrt_status launch_step();
    flexrt_status launch_stage(int stage);
    flexrt_status read_acc(int slot, SimAcc &a);
    void free_retired();

    EngineConfig cfg_{};
    int device_ = 0;
    cudaStream_t st_ = nullptr;
    bool own_stream_ = false;
    std::string err_;
    flexrt_status latched_ = FLEXRT_OK;

    Ctl *ctl_ = nullptr;
    SimDev *sims_ = nullptr;
    SimAcc *acc_ = nullptr;
    void *qmem_ = nullptr;
    Queue q_[2]{};
    Cells cells_{};
    Emitters em_{};
    Ranges rg_{};
    MergeWork mw_{};
    void *mwmem_ = nullptr;
    const int4 *pixtab_ = nullptr;
    int ltab_ = 0;
    int em_cap_ = 0;
    long long qcap_ = 0;       // allocated queue slots (capacity plus run-tail margin)
    RangeAllocator cell_alloc_, em_alloc_;
    std::vector<Slot> slots_;
    long long steps_taken_ = 0;

    int march_agg_ = 0, march_minb_ = 3, march_blocks_ = 1, march_threads_ = 256, march_slab_ = OUT_SLAB;
    int chem_blocks_ = 1, emit_blocks_ = 1, sm_count_ = 1;

    int32_t *h_err_ = nullptr;     // the last step's queue counts, parity and error word
    double *h_stage_ = nullptr;
    double *h_nh_ = nullptr;       // pinned staging of a member's n_H (engines of several members)
    void *h_fields_ = nullptr;     // pinned staging of the fields read-back, grown on demand
    size_t h_fields_bytes_ = 0;
    cudaEvent_t ev_nh_ = nullptr;  // its upload has been consumed
    long long q_used_ = 0;         // live rays after the last step the host has seen complete
    cudaEvent_t ev_err_ = nullptr, ev_stage_ = nullptr;
    MergeSide mside_{nullptr, nullptr, nullptr};   // merging engines: the rotation pass's stream
    bool err_pending_ = false;

    bool profiling_ = false;
    std::vector<cudaEvent_t> ev_pool_;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_k_[4];
    double rays_at_profile_ = 0.0;

    cudaGraphExec_t graph_ = nullptr;
    bool graph_dirty_ = true;
    bool mid_step_ = false;                 // between the two stages of a staged step

    std::unordered_map<void *, size_t> alloc_sizes_;   // live device allocations
    long long alloc_bytes_ = 0;
};

}  // namespace frt
