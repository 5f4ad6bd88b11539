// frt_static.cu -- the one-step traversal probe without device allocation.
//
// flexrt_probe_traverse stages its host inputs and outputs in device buffers
// it allocates on every call.  This variant keeps that staging in one fixed
// file-scope device array instead, so a call never allocates or frees device
// memory.  It launches the same traversal kernel.
//
// The array lives on every GPU that loads the library until the process
// exits.  In host code `g_stage` names a host-side stand-in, not a device
// address: its device address is looked up once per device (with that device
// current) with cudaGetSymbolAddress, kept for the life of the process and
// handed to the kernel.  A device reset between calls would leave the kept
// address stale; callers must not reset the device between calls.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/flexrt.h"
#include "frt_launch.h"

namespace {

constexpr long long kMaxRays = FLEXRT_STATIC_MAX_RAYS;
// per-ray staging, each region a multiple of 256 bytes for kMaxRays rays
constexpr size_t kP0 = 0;                                   // int64[3]
constexpr size_t kDir = kP0 + kMaxRays * 3 * sizeof(long long);   // int32[3]
constexpr size_t kCells = kDir + kMaxRays * 3 * sizeof(int32_t);  // int32[4][3]
constexpr size_t kDs = kCells + kMaxRays * 12 * sizeof(int32_t);  // float[4]
constexpr size_t kNseg = kDs + kMaxRays * 4 * sizeof(float);      // int32
constexpr size_t kEsc = kNseg + kMaxRays * sizeof(int32_t);       // int32
constexpr size_t kBytes = kEsc + kMaxRays * sizeof(int32_t);
static_assert(kDir % 256 == 0 && kCells % 256 == 0 && kDs % 256 == 0 && kNseg % 256 == 0 && kEsc % 256 == 0,
              "staging regions must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_stage[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

// device address of g_stage on the current device (resolved on first use)
cudaError_t stage_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stage);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

flexrt_status fail(flexrt_status s, const std::string &m) {
    frt::set_free_error(m);
    return s;
}

}  // namespace

extern "C" flexrt_status flexrt_probe_traverse_static(int64_t n, const int64_t *p0, const int32_t *dir,
                                                      const flexrt_grid *g, int32_t *cells, float *ds,
                                                      int32_t *nseg, int32_t *escaped) {
    if (n < 0 || !g || (n && (!p0 || !dir || !cells || !ds || !nseg || !escaped)))
        return fail(FLEXRT_E_INVALID, "flexrt_probe_traverse_static: bad arguments");
    if (n > kMaxRays)
        return fail(FLEXRT_E_CAPACITY, "flexrt_probe_traverse_static: n = " + std::to_string(n) +
                                           " exceeds the fixed maximum of " + std::to_string(kMaxRays) +
                                           " rays per call (FLEXRT_STATIC_MAX_RAYS)");
    for (int64_t i = 0; i < 3 * n; ++i)
        if (dir[i] > (1 << 21) || dir[i] < -(1 << 21) || p0[i] > (1LL << 31) - (1LL << 22) ||
            p0[i] < -(1LL << 31) + (1LL << 22))
            return fail(FLEXRT_E_INVALID, "flexrt_probe_traverse_static: |d| > 2^21 or |p0| >= 2^31 - 2^22");
    if (n == 0) return FLEXRT_OK;
    unsigned char *base = nullptr;
    cudaError_t e = stage_address(&base);
    if (e != cudaSuccess) return fail(FLEXRT_E_CUDA, std::string("static staging address: ") + cudaGetErrorString(e));
    long long *d_p0 = reinterpret_cast<long long *>(base + kP0);
    int32_t *d_dir = reinterpret_cast<int32_t *>(base + kDir);
    int32_t *d_cells = reinterpret_cast<int32_t *>(base + kCells);
    float *d_ds = reinterpret_cast<float *>(base + kDs);
    int32_t *d_nseg = reinterpret_cast<int32_t *>(base + kNseg);
    int32_t *d_esc = reinterpret_cast<int32_t *>(base + kEsc);
    // the array keeps the previous call's contents: reset what the kernel
    // leaves untouched for rays with fewer than four segments
    if ((e = cudaMemcpy(d_p0, p0, 3 * n * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_dir, dir, 3 * n * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(d_cells, 0xff, 12 * n * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(d_ds, 0, 4 * n * sizeof(float))) != cudaSuccess)
        return fail(FLEXRT_E_CUDA, std::string("static staging upload: ") + cudaGetErrorString(e));
    e = frt::launch_probe_traverse(n, d_p0, d_dir, g->nx, g->ny, g->nz, d_cells, d_ds, d_nseg, d_esc, 0);
    if (e != cudaSuccess) return fail(FLEXRT_E_CUDA, std::string("traversal kernel: ") + cudaGetErrorString(e));
    if ((e = cudaMemcpy(cells, d_cells, 12 * n * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(ds, d_ds, 4 * n * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(nseg, d_nseg, n * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(escaped, d_esc, n * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(FLEXRT_E_CUDA, std::string("static staging download: ") + cudaGetErrorString(e));
    return FLEXRT_OK;
}
