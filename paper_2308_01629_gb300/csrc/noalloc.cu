// noalloc.cu -- LR-style binning whose scratch memory is a fixed array that
// the library itself holds in device memory, for callers that cannot
// allocate device memory.
//
// The radix sort behind gs_bin_low needs scratch beyond its inputs and
// outputs (a second key/index buffer pair and a digit histogram).  Here that
// scratch is one static __device__ array of fixed size.  Every GPU that loads
// this library keeps the array (GS_STATIC_BIN_SCRATCH_BYTES) until the
// process exits.  All calls on one device share it: calls that overlap on the
// GPU race and corrupt each other's results.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = GS_STATIC_BIN_MAX_POINTS;
constexpr size_t kHistWords = 256 * 160;   // digit histogram of up to 160 sort tiles
constexpr size_t kWords = 4 * (size_t)kMaxPoints + kHistWords;
static_assert(kWords * sizeof(uint32_t) == GS_STATIC_BIN_SCRATCH_BYTES, "scratch size in gs.h is out of date");

// Layout: keys[2][kMaxPoints], indices[2][kMaxPoints], histogram[kHistWords].
// Every word a call reads it has written first in the same call, so nothing
// needs clearing between calls.
static __device__ __align__(256) uint32_t g_bin_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device with that device current.
int scratch_on_current_device(uint32_t** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace

extern "C" int gs_bin_points_static(const float* pos4, int64_t n, const gs_grid_info* grid, uint32_t* sorted_index,
                                    uint32_t* cell_start, void* cuda_stream)
{
    if (!grid || !cell_start || n < 0) return GS_ERR_ARG;
    if (n > kMaxPoints) return GS_ERR_CAPACITY;
    if (n > 0 && (!pos4 || !sorted_index)) return GS_ERR_ARG;
    if (n > 0 && (reinterpret_cast<uintptr_t>(pos4) & 15u) != 0) return GS_ERR_ARG;   // float4 records
    // uint32 words: the cell starts are written by a kernel, the sorted
    // indices by a copy
    if ((reinterpret_cast<uintptr_t>(cell_start) & 3u) != 0) return GS_ERR_ARG;
    if (n > 0 && (reinterpret_cast<uintptr_t>(sorted_index) & 3u) != 0) return GS_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (grid->dims[k] < 1 || grid->dims[k] > (1 << 20)) return GS_ERR_ARG;   // as gs_create
    const int64_t n_cell = (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2];
    if (n_cell != grid->n_cell || n_cell >= 0xffffffffLL || !(grid->inv_h > 0.0f)) return GS_ERR_ARG;
    if (gs_sort_hist_words(n) > kHistWords) return GS_ERR_CAPACITY;

    uint32_t* base = nullptr;
    int st = scratch_on_current_device(&base);
    if (st != GS_OK) return st;

    GridDev g;
    g.ox = grid->origin[0];
    g.oy = grid->origin[1];
    g.oz = grid->origin[2];
    g.h = grid->h;
    g.inv_h = grid->inv_h;
    g.dx = grid->dims[0];
    g.dy = grid->dims[1];
    g.dz = grid->dims[2];

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t* keys[2] = {base, base + kMaxPoints};
    uint32_t* vals[2] = {base + 2 * kMaxPoints, base + 3 * kMaxPoints};
    uint32_t* hist = base + 4 * kMaxPoints;
    int64_t launches = 0;
    int which = 0;
    if (gs_launch_cell_keys(s, reinterpret_cast<const float4*>(pos4), n, g, 0, keys[0], vals[0], &launches) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    if (gs_radix_sort(s, keys, vals, &which, hist, n, gs_key_bits(n_cell), &launches) != cudaSuccess)
        return GS_ERR_CUDA;
    if (n > 0 && cudaMemcpyAsync(sorted_index, vals[which], (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                 s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (gs_launch_cell_start(s, keys[which], n, n_cell, cell_start, &launches) != cudaSuccess) return GS_ERR_CUDA;
    return GS_OK;
}
