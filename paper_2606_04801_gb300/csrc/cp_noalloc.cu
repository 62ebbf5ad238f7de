// Backward scatter that allocates nothing: cubical_persistence_backward_noalloc.
//
// Some callers cannot allocate device memory at all: code inside another
// framework's callbacks that has no handle on its allocator, or deployments
// whose device memory is fully reserved up front by another component.
// Those callers can still pass their own inputs and output, but not a
// workspace.  This entry point computes the same gradient as
// cubical_persistence_backward with its double-precision accumulators in a
// fixed array that is part of this library's device image instead of a
// caller-provided workspace.
//
// The array holds kNoallocMaxPixels doubles (32 MiB); every GPU that loads
// the library keeps it until the process exits.  All calls share it: a call
// clears the part it uses before accumulating, and two calls whose work
// overlaps on the GPU (for example on two streams without ordering between
// them) race on it.
#include <mutex>

#include "cp_common.cuh"
#include "cp_kernels.h"

namespace cp {
namespace {

constexpr int64_t kNoallocMaxPixels = int64_t(1) << 22;
constexpr int kT = 256;

static __device__ __align__(256) double g_noalloc_acc[kNoallocMaxPixels];

__global__ void k_noalloc_clear(double* acc, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) acc[i] = 0.0;
}

__global__ void k_noalloc_scatter(const cp_pair* __restrict__ pairs, int64_t n, const float* __restrict__ gb,
                                  const float* __restrict__ gd, const int64_t* __restrict__ offs, double* acc,
                                  int64_t n_pixels) {
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT) {
        const cp_pair& p = pairs[i];
        int64_t off = offs ? offs[p.item] : 0;
        if (p.birth_pixel >= 0) {
            int64_t q = off + p.birth_pixel;
            if (q >= 0 && q < n_pixels) atomicAdd(acc + q, double(gb[i]));
        }
        if (p.death_pixel >= 0) {
            int64_t q = off + p.death_pixel;
            if (q >= 0 && q < n_pixels) atomicAdd(acc + q, double(gd[i]));
        }
    }
}

__global__ void k_noalloc_round(const double* __restrict__ acc, float* __restrict__ grad, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * kT + threadIdx.x; i < n; i += int64_t(gridDim.x) * kT)
        grad[i] = float(acc[i]);
}

// Device address of g_noalloc_acc per device, looked up once per device with
// that device current.  In host code the array's name only stands for the
// host-side shadow of the symbol, never for device memory.  The cache is
// keyed by device ordinal, so a cudaDeviceReset of a device after its first
// call here is not supported (the module would reload at another address).
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};

int noalloc_setup(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p) return CP_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CP_OK;
}

int grid_for(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    int64_t cap = int64_t(device_sm_count()) * 8;
    return int(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace cp

extern "C" int64_t cubical_persistence_backward_noalloc_max_pixels(void) { return cp::kNoallocMaxPixels; }

extern "C" int cubical_persistence_backward_noalloc(const cp_pair* d_pairs, int64_t n_pairs, const float* d_grad_birth,
                                                    const float* d_grad_death, const int64_t* d_item_offsets,
                                                    float* d_grad_image, int64_t n_pixels, void* stream) {
    using namespace cp;
    if (n_pairs < 0 || n_pixels <= 0 || !d_grad_image) return CP_ERR_ARG;
    if (n_pairs > 0 && (!d_pairs || !d_grad_birth || !d_grad_death)) return CP_ERR_ARG;
    if (n_pixels > kNoallocMaxPixels) return CP_ERR_CAPACITY;
    double* acc = nullptr;
    int rc = noalloc_setup(&acc);
    if (rc != CP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_clear<<<grid_for(n_pixels), kT, 0, s>>>(acc, n_pixels);
    if (n_pairs > 0)
        k_noalloc_scatter<<<grid_for(n_pairs), kT, 0, s>>>(d_pairs, n_pairs, d_grad_birth, d_grad_death, d_item_offsets,
                                                           acc, n_pixels);
    k_noalloc_round<<<grid_for(n_pixels), kT, 0, s>>>(acc, d_grad_image, n_pixels);
    note_launches(n_pairs > 0 ? 3 : 2);
    return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ERR_CUDA;
}
