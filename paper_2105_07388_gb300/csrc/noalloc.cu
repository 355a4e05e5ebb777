// re_sketch_apply_noalloc: the Gaussian sketch step of re_sketch_apply (FP32
// right sketch, split-K left sketch) for callers that may not allocate device
// memory.  Its scratch -- the generated X columns and the left sketch's split-K
// partial sums -- lives in one file-scope __device__ array instead of a
// handle's workspace, so the call needs no handle, no cudaMalloc/cudaFree and
// no allocating library routine.
//
// Every GPU that loads this library holds the array (16 MiB) until the
// process exits.  All calls on a device share it, so calls that overlap on
// the GPU (different streams, or different host threads) race on it and must
// be serialised by the caller.  Nothing in it needs to start at zero: each call
// writes every scratch element it later reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr size_t kScratchFloats = (size_t)4 << 20;          // 4 Mi floats = 16 MiB

__device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device;
// in host code the symbol itself is only a host-side stand-in).
cudaError_t scratch_on_current_device(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace re

// Device that holds `p` (device memory or managed memory), or -1.
static int device_of(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return -1;
    return a.device;
}

extern "C" int re_sketch_apply_noalloc(const void* A, int dtype, int64_t m, int64_t n, int64_t ld,
                                       int col0, int s, uint64_t seed, float* AX, int64_t ld_ax,
                                       double* core, int64_t ld_core, void* stream) {
    using namespace re;
    if (!A || !AX) return set_last_error(RE_ERR_ARG, "NULL argument");
    if (dtype != RE_F32 && dtype != RE_F64) return set_last_error(RE_ERR_ARG, "dtype must be RE_F32 or RE_F64");
    if (m <= 0 || n <= 0 || ld < n) return set_last_error(RE_ERR_ARG, "bad shape or ld < n");
    if (m > INT32_MAX || n > INT32_MAX) return set_last_error(RE_ERR_ARG, "dimension too large");
    if (col0 < 0 || col0 % 8 != 0 || s <= 0 || s % 8 != 0)
        return set_last_error(RE_ERR_ARG, "col0 and s must be multiples of 8, s > 0");
    if (ld_ax < col0 + s) return set_last_error(RE_ERR_ARG, "ld_ax < col0 + s");
    if (core && ld_core < col0 + s) return set_last_error(RE_ERR_ARG, "ld_core < col0 + s");
    // the kernels run on the device that holds A; AX and core must live there too
    const int dev = device_of(A);
    if (dev < 0) return set_last_error(RE_ERR_ARG, "A is not device memory");
    if (device_of(AX) != dev || (core && device_of(core) != dev))
        return set_last_error(RE_ERR_ARG, "A, AX and core must be device memory of one device");
    MatView V;
    V.ptr = A;
    V.dtype = dtype;
    V.trans = m < n;
    V.rows = std::max(m, n);
    V.cols = std::min(m, n);
    V.ld = ld;
    const int c1 = col0 + s;
    // scratch: X columns (cols x s), then the split-K partials of the larger left block
    const size_t x_floats = ((size_t)V.cols * s + 63) / 64 * 64;
    size_t part_floats = 0;
    if (core) {
        part_floats = left_part_floats(V.rows, 2 * c1, s);
        if (col0 > 0) part_floats = std::max(part_floats, left_part_floats(V.rows, 2 * s, col0));
    }
    if (x_floats + part_floats > kScratchFloats)
        return set_last_error(RE_ERR_ARG,
                              "re_sketch_apply_noalloc: problem needs more than the 16 MiB static "
                              "scratch (min(m,n)*s + left-sketch partials > 4 Mi floats)");
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, cudaGetErrorString(e));
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
        return set_last_error(RE_ERR_CUDA, cudaGetErrorString(e));
    float* scratch = nullptr;
    e = scratch_on_current_device(&scratch);
    if (e == cudaSuccess) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        float* X = scratch;
        float* part = scratch + x_floats;
        e = launch_gauss_x(seed, V.cols, col0, s, X, s, st);
        if (e == cudaSuccess) e = launch_right_simt(V, X, s, s, AX + col0, ld_ax, st);
        if (e == cudaSuccess && core && col0 > 0)
            e = launch_left(seed, AX, ld_ax, V.rows, 2 * col0, 2 * s, 0, col0, part, part_floats, core, ld_core, st);
        if (e == cudaSuccess && core)
            e = launch_left(seed, AX, ld_ax, V.rows, 0, 2 * c1, col0, s, part, part_floats, core, ld_core, st);
    }
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, cudaGetErrorString(e));
    return RE_OK;
}
