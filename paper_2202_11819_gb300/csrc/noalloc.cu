// jac_residual_dense_noalloc: the residual of a dense grid held by the
// caller, computed without allocating any memory.
//
// Why: some callers cannot call cudaMalloc at the point where they need the
// residual -- code running while a memory pool is locked or being resized, a
// framework that forbids allocations inside its step, or a host-side
// callback that must not block on the allocator. The regular entry points
// allocate their scratch (the per-CTA partial sums) inside a context; this
// one keeps that scratch in a fixed-size array inside the library.
//
// Scratch: kNoAllocMaxPartials doubles (512 KiB) in a file-scope static
// __device__ array. Every GPU that loads the library holds this array until
// the process exits. Each call writes every partial slot it later reads, so
// nothing needs clearing between calls; the array keeps the last call's
// contents. All calls share the one array, so calls whose kernels overlap on
// the GPU (on different streams, or from several host threads) race and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "arith.cuh"
#include "jacobi3d.h"

namespace {

constexpr int kNoAllocMaxPartials = 1 << 16;
constexpr int kDX = 32;
constexpr int kDY = 8;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

// Value at (x, y, k) of the dense grid, or the Dirichlet value of the face
// that (x, y, k) lies outside of (at most one coordinate is outside).
template <typename T>
__device__ __forceinline__ double dense_at(const T* u, int nx, int ny, int nz, const double* bc, int x, int y, int k)
{
    if (x < 0) return (double)(T)bc[0];
    if (x >= nx) return (double)(T)bc[1];
    if (y < 0) return (double)(T)bc[2];
    if (y >= ny) return (double)(T)bc[3];
    if (k < 0) return (double)(T)bc[4];
    if (k >= nz) return (double)(T)bc[5];
    return (double)u[(int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * k)];
}

// One partial per CTA: the sum over its 32 x 8 columns (all k) of L^2, L the
// exact Laplacian term rounded once, accumulated with fused multiply-adds
// (acc = fma(L, L, acc)); fixed order (per thread over k, then a fixed tree),
// so the result is deterministic.
template <typename T>
__global__ void __launch_bounds__(kDX * kDY)
k_residual_dense(const T* u, int nx, int ny, int nz, double b0, double b1, double b2, double b3, double b4, double b5,
                 double* partials)
{
    __shared__ double red[kDX * kDY];
    const double bc[6] = {b0, b1, b2, b3, b4, b5};
    const int x = blockIdx.x * kDX + threadIdx.x;
    const int y = blockIdx.y * kDY + threadIdx.y;
    double acc = 0.0;
    if (x < nx && y < ny) {
        double zm = dense_at(u, nx, ny, nz, bc, x, y, -1);
        double c = dense_at(u, nx, ny, nz, bc, x, y, 0);
        for (int k = 0; k < nz; ++k) {
            const double zp = dense_at(u, nx, ny, nz, bc, x, y, k + 1);
            const double L = jac::laplacian_exact(c, dense_at(u, nx, ny, nz, bc, x - 1, y, k),
                                                  dense_at(u, nx, ny, nz, bc, x + 1, y, k),
                                                  dense_at(u, nx, ny, nz, bc, x, y - 1, k),
                                                  dense_at(u, nx, ny, nz, bc, x, y + 1, k), zm, zp);
            acc = fma(L, L, acc);
            zm = c;
            c = zp;
        }
    }
    const int tid = threadIdx.y * kDX + threadIdx.x;
    red[tid] = acc;
    __syncthreads();
    for (int s = kDX * kDY / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_sum_dense_partials(const double* partials, int n, double* out)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = acc + partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

// Makes `dev` the calling thread's current device for the guard's lifetime
// and puts the caller's device back on every return path.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t enter(int dev)
    {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess || prev == dev) return e;
        e = cudaSetDevice(dev);
        switched = e == cudaSuccess;
        return e;
    }
    ~DeviceGuard()
    {
        if (switched) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int jac_residual_dense_noalloc(const void* u, int32_t dtype, int64_t nx, int64_t ny, int64_t nz,
                                          const double bc[6], double* out, void* stream)
{
    if (!u || !out || !bc) return JAC_EINVAL;
    if (dtype != JAC_F64 && dtype != JAC_F32) return JAC_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) return JAC_EINVAL;
    for (int f = 0; f < 6; ++f)
        if (!std::isfinite(bc[f])) return JAC_EINVAL;
    const int64_t gx = (nx + kDX - 1) / kDX, gy = (ny + kDY - 1) / kDY;
    if (gx * gy > kNoAllocMaxPartials || gy > 65535) return JAC_EINVAL;  // beyond the fixed scratch
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = s ? cudaStreamGetDevice(s, &dev) : cudaGetDevice(&dev);
    if (e != cudaSuccess) return JAC_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return JAC_EINVAL;
    // the symbol lookup and the launches need the stream's device current;
    // the caller's current device is restored on return
    DeviceGuard guard;
    if (guard.enter(dev) != cudaSuccess) return JAC_ECUDA;
    double* partials;
    {
        // first call on a device: look up the device address of the static
        // array (the host-side name is only a stand-in for it)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_partials_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return JAC_ECUDA;
            g_partials_addr[dev] = (double*)p;
        }
        partials = g_partials_addr[dev];
    }
    const dim3 grid((unsigned)gx, (unsigned)gy, 1), block(kDX, kDY, 1);
    if (dtype == JAC_F64)
        k_residual_dense<double><<<grid, block, 0, s>>>((const double*)u, (int)nx, (int)ny, (int)nz, bc[0], bc[1],
                                                        bc[2], bc[3], bc[4], bc[5], partials);
    else
        k_residual_dense<float><<<grid, block, 0, s>>>((const float*)u, (int)nx, (int)ny, (int)nz, bc[0], bc[1],
                                                       bc[2], bc[3], bc[4], bc[5], partials);
    if (cudaGetLastError() != cudaSuccess) return JAC_ECUDA;
    k_sum_dense_partials<<<1, 256, 0, s>>>(partials, (int)(gx * gy), out);
    if (cudaGetLastError() != cudaSuccess) return JAC_ECUDA;
    return JAC_OK;
}
