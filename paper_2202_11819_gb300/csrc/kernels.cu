// Kernels of libjacobi3d (sm_103a).
//
// The paper's per-iteration kernel flow (Section II-A, Figs. 1 and 3;
// Section III-D1) is: pack the six boundary faces of a block into send
// buffers, exchange them with the neighbours, unpack the received halos into
// the ghost layer, update the whole block. Here:
//   k_pack_face / k_unpack_face   one face per launch (the unfused flow),
//   k_pack6 / k_unpack6           the six faces fused into one launch with one
//                                 thread per cell of the LARGEST face, each
//                                 thread visiting the six faces in turn
//                                 (the mapping Section III-D1 found faster
//                                 than one thread per cell of all faces),
//   k_stencil_block               the update of one block from its own ghost
//                                 layer (unfused flow),
//   k_fused_step                  unpack + update + pack of every block in one
//                                 launch (strategy C): ghost values are read
//                                 straight from the neighbouring blocks,
//   k_persistent                  all blocks and all iterations in one launch,
//                                 each tile waiting only for the previous
//                                 iteration of its own and neighbouring blocks
//                                 (the device form of the per-iteration
//                                 reference numbers of Section II-A),
//   k_residual / k_sum_partials   the residual norm, deterministic order,
//   k_scatter / k_gather          dense x-fastest arrays <-> block storage.
#include <cuda_runtime.h>

#include <cstdint>

#include "arith.cuh"
#include "jac_common.cuh"
#include "launch.h"

namespace jac {

// Tile of the z-marching update: 32 x 8 threads, each thread owning VX
// columns spaced 32 apart, so one tile covers 64 x 8 columns of a block.
constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kVX = 2;
constexpr int kTW = kTX * kVX;
constexpr int kSW = kTW + 2;  // shared row with one halo cell on each side
constexpr int kSmemCells = (kTY + 2) * kSW;

template <typename T>
__device__ __forceinline__ int64_t cell_index(const BlockDesc& d, int p, int x, int y, int k)
{
    return d.off[p] + (int64_t)(k + 1) * d.plane + (int64_t)(y + 1) * d.pitch + Layout<T>::OX + x;
}

template <typename T, bool CG>
__device__ __forceinline__ T ld(const T* p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Value of cell (x, y, k) of block d in buffer p, where at most one coordinate
// may lie one step outside the block. PULL: an outside cell is read from the
// neighbouring block's interior (or is the Dirichlet value at the global
// boundary). Otherwise it is read from the block's own ghost layer.
template <typename T, bool PULL, bool CG>
__device__ __forceinline__ T load_cell(const T* __restrict__ pool, const BlockDesc* __restrict__ desc,
                                       const BlockDesc& d, int p, int x, int y, int k)
{
    if constexpr (PULL) {
        int f = -1;
        if (x < 0) f = 0;
        else if (x >= d.ext[0]) f = 1;
        else if (y < 0) f = 2;
        else if (y >= d.ext[1]) f = 3;
        else if (k < 0) f = 4;
        else if (k >= d.ext[2]) f = 5;
        if (f >= 0) {
            const int nb = d.nbr[f];
            if (nb < 0) return (T)d.bc[f];
            const BlockDesc& n = desc[nb];
            int xx = x, yy = y, kk = k;
            switch (f) {
                case 0: xx = n.ext[0] - 1; break;
                case 1: xx = 0; break;
                case 2: yy = n.ext[1] - 1; break;
                case 3: yy = 0; break;
                case 4: kk = n.ext[2] - 1; break;
                default: kk = 0; break;
            }
            return ld<T, CG>(pool + cell_index<T>(n, p, xx, yy, kk));
        }
    }
    return ld<T, CG>(pool + cell_index<T>(d, p, x, y, k));
}

template <typename T, int ARITH>
__device__ __forceinline__ T mean7(T c, T xm, T xp, T ym, T yp, T zm, T zp)
{
    if constexpr (sizeof(T) == 4) {
        return mean7_seq_f32(c, xm, xp, ym, yp, zm, zp);
    } else if constexpr (ARITH == 1) {
        return mean7_exact(c, xm, xp, ym, yp, zm, zp);
    } else {
        return mean7_seq(c, xm, xp, ym, yp, zm, zp);
    }
}

// The z-marching update of one tile (x0..x0+63, y0..y0+7, all k) of block b:
// reads buffer p, writes the interior of buffer p^1. The current plane of the
// tile plus a one-cell halo ring sits in shared memory; the planes below and
// above are carried in registers.
template <typename T, int ARITH, bool PULL, bool CG>
__device__ void update_tile(T* __restrict__ pool, const BlockDesc* __restrict__ desc, int b, int p,
                            int x0, int y0, T* sm)
{
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y = y0 + ty;
    const bool yin = y < by;
    T zm[kVX], c[kVX], zp[kVX];
#pragma unroll
    for (int v = 0; v < kVX; ++v) {
        const int x = x0 + tx + kTX * v;
        if (yin && x < bx) {
            zm[v] = load_cell<T, PULL, CG>(pool, desc, d, p, x, y, -1);
            c[v] = ld<T, CG>(pool + cell_index<T>(d, p, x, y, 0));
        } else {
            zm[v] = T(0);
            c[v] = T(0);
        }
    }
    for (int k = 0; k < bz; ++k) {
#pragma unroll
        for (int v = 0; v < kVX; ++v) {
            const int x = x0 + tx + kTX * v;
            if (yin && x < bx) {
                zp[v] = (k + 1 < bz) ? ld<T, CG>(pool + cell_index<T>(d, p, x, y, k + 1))
                                     : load_cell<T, PULL, CG>(pool, desc, d, p, x, y, bz);
            } else {
                zp[v] = T(0);
            }
            // own slot: the cell itself, or the +x / +y halo when the tile
            // overhangs the block edge by exactly that cell
            T s = T(0);
            if (yin && x < bx) s = c[v];
            else if (yin && x == bx) s = load_cell<T, PULL, CG>(pool, desc, d, p, x, y, k);
            else if (y == by && x < bx) s = load_cell<T, PULL, CG>(pool, desc, d, p, x, y, k);
            sm[(ty + 1) * kSW + tx + kTX * v + 1] = s;
        }
        if (ty == 0) {  // row y0 - 1
#pragma unroll
            for (int v = 0; v < kVX; ++v) {
                const int x = x0 + tx + kTX * v;
                sm[tx + kTX * v + 1] = x < bx ? load_cell<T, PULL, CG>(pool, desc, d, p, x, y0 - 1, k) : T(0);
            }
        }
        if (ty == kTY - 1 && y0 + kTY <= by) {  // row y0 + 8 (inside or +y halo)
#pragma unroll
            for (int v = 0; v < kVX; ++v) {
                const int x = x0 + tx + kTX * v;
                sm[(kTY + 1) * kSW + tx + kTX * v + 1] =
                    x < bx ? load_cell<T, PULL, CG>(pool, desc, d, p, x, y0 + kTY, k) : T(0);
            }
        }
        if (tx == 0) sm[(ty + 1) * kSW] = yin ? load_cell<T, PULL, CG>(pool, desc, d, p, x0 - 1, y, k) : T(0);
        if (tx == kTX - 1 && x0 + kTW <= bx)
            sm[(ty + 1) * kSW + kTW + 1] = yin ? load_cell<T, PULL, CG>(pool, desc, d, p, x0 + kTW, y, k) : T(0);
        __syncthreads();
#pragma unroll
        for (int v = 0; v < kVX; ++v) {
            const int x = x0 + tx + kTX * v;
            if (yin && x < bx) {
                const int sc = (ty + 1) * kSW + tx + kTX * v + 1;
                const T out = mean7<T, ARITH>(c[v], sm[sc - 1], sm[sc + 1], sm[sc - kSW], sm[sc + kSW], zm[v], zp[v]);
                pool[cell_index<T>(d, p ^ 1, x, y, k)] = out;
            }
            zm[v] = c[v];
            c[v] = zp[v];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- kernels

template <typename T, int ARITH>
__global__ void __launch_bounds__(kTX * kTY) k_stencil_block(T* pool, const BlockDesc* desc, int b, int p)
{
    __shared__ T sm[kSmemCells];
    update_tile<T, ARITH, false, false>(pool, desc, b, p, blockIdx.x * kTW, blockIdx.y * kTY, sm);
}

template <typename T, int ARITH>
__global__ void __launch_bounds__(kTX * kTY) k_fused_step(T* pool, const BlockDesc* desc, const TileUnit* units, int p)
{
    __shared__ T sm[kSmemCells];
    const TileUnit u = units[blockIdx.x];
    update_tile<T, ARITH, true, false>(pool, desc, u.block, p, u.x0, u.y0, sm);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p)
{
    return *(const volatile int32_t*)p;
}

// Persistent form. Work unit w = (iteration t = w / U, tile u = w % U) is
// taken in increasing w from one global counter, so every unit a CTA waits on
// was taken earlier by a CTA that is already running: the launch cannot
// deadlock whatever number of CTAs is resident. Before computing (t, tile of
// block b), the CTA waits until b and its six neighbours have each finished
// all their tiles of iteration t-1 (done[n] >= t * ntiles[n]): that covers
// both the halo it reads (buffer p) and every reader of the region it
// overwrites (buffer p^1 held iteration t-1). Every wait is bounded.
template <typename T, int ARITH>
__global__ void __launch_bounds__(kTX * kTY) k_persistent(T* pool, const BlockDesc* desc, const TileUnit* units,
                                                          int nunits, int p0, int64_t n_iters, uint32_t* done,
                                                          unsigned long long* work, DeviceStatus* st,
                                                          int64_t wait_ns, int hold_block, int64_t hold_after)
{
    __shared__ T sm[kSmemCells];
    __shared__ long long s_w;
    __shared__ int s_stop;
    const long long total = (long long)n_iters * nunits;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    for (;;) {
        if (lead) {
            long long w = ld_volatile(&st->abort) ? total : (long long)atomicAdd(work, 1ull);
            s_w = w;
            int stop = 0;
            if (w < total) {
                const int t = (int)(w / nunits);
                const int b = units[w % nunits].block;
                if (t > 0) {
                    const uint64_t t0 = global_ns();
                    for (int f = -1; f < 6 && !stop; ++f) {
                        const int n = f < 0 ? b : desc[b].nbr[f];
                        if (n < 0) continue;
                        const uint32_t need = (uint32_t)t * (uint32_t)desc[n].ntiles;
                        unsigned ns = 32;
                        while (ld_acquire(done + n) < need) {
                            if (ld_volatile(&st->abort)) {
                                stop = 1;
                                break;
                            }
                            if ((int64_t)(global_ns() - t0) > wait_ns) {
                                if (atomicCAS(&st->err, kErrNone, kErrTimeout) == kErrNone) {
                                    st->where_block = n;
                                    st->where_iter = t;
                                }
                                atomicExch(&st->abort, 1);
                                stop = 1;
                                break;
                            }
                            __nanosleep(ns);
                            ns = ns < 1024 ? ns * 2 : ns;
                        }
                    }
                    __threadfence();
                }
            }
            s_stop = stop;
        }
        __syncthreads();
        const long long w = s_w;
        if (w >= total || s_stop) break;
        const int t = (int)(w / nunits);
        const TileUnit u = units[w % nunits];
        update_tile<T, ARITH, true, true>(pool, desc, u.block, (p0 + t) & 1, u.x0, u.y0, sm);
        __syncthreads();
        if (lead && !(u.block == hold_block && t >= hold_after)) {
            __threadfence();
            atomicAdd(done + u.block, 1u);
        }
    }
}

// Residual: sum over the tile of L^2, L = xm+xp+ym+yp+zm+zp-6c exact, one
// partial per CTA in a fixed order (per thread over k, then a fixed tree).
template <typename T>
__global__ void __launch_bounds__(kTX * kTY) k_residual(const T* pool, const BlockDesc* desc, const TileUnit* units,
                                                        int p, double* partials)
{
    __shared__ T sm[kSmemCells];
    __shared__ double red[kTX * kTY];
    const TileUnit u = units[blockIdx.x];
    const BlockDesc& d = desc[u.block];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = u.x0, y0 = u.y0;
    const int y = y0 + ty;
    const bool yin = y < by;
    double acc = 0.0;
    T zm[kVX], c[kVX], zp[kVX];
#pragma unroll
    for (int v = 0; v < kVX; ++v) {
        const int x = x0 + tx + kTX * v;
        if (yin && x < bx) {
            zm[v] = load_cell<T, true, false>(pool, desc, d, p, x, y, -1);
            c[v] = pool[cell_index<T>(d, p, x, y, 0)];
        } else {
            zm[v] = T(0);
            c[v] = T(0);
        }
    }
    for (int k = 0; k < bz; ++k) {
#pragma unroll
        for (int v = 0; v < kVX; ++v) {
            const int x = x0 + tx + kTX * v;
            if (yin && x < bx)
                zp[v] = (k + 1 < bz) ? pool[cell_index<T>(d, p, x, y, k + 1)]
                                     : load_cell<T, true, false>(pool, desc, d, p, x, y, bz);
            else
                zp[v] = T(0);
            T s = T(0);
            if (yin && x < bx) s = c[v];
            else if (yin && x == bx) s = load_cell<T, true, false>(pool, desc, d, p, x, y, k);
            else if (y == by && x < bx) s = load_cell<T, true, false>(pool, desc, d, p, x, y, k);
            sm[(ty + 1) * kSW + tx + kTX * v + 1] = s;
        }
        if (ty == 0) {
#pragma unroll
            for (int v = 0; v < kVX; ++v) {
                const int x = x0 + tx + kTX * v;
                sm[tx + kTX * v + 1] = x < bx ? load_cell<T, true, false>(pool, desc, d, p, x, y0 - 1, k) : T(0);
            }
        }
        if (ty == kTY - 1 && y0 + kTY <= by) {
#pragma unroll
            for (int v = 0; v < kVX; ++v) {
                const int x = x0 + tx + kTX * v;
                sm[(kTY + 1) * kSW + tx + kTX * v + 1] =
                    x < bx ? load_cell<T, true, false>(pool, desc, d, p, x, y0 + kTY, k) : T(0);
            }
        }
        if (tx == 0) sm[(ty + 1) * kSW] = yin ? load_cell<T, true, false>(pool, desc, d, p, x0 - 1, y, k) : T(0);
        if (tx == kTX - 1 && x0 + kTW <= bx)
            sm[(ty + 1) * kSW + kTW + 1] = yin ? load_cell<T, true, false>(pool, desc, d, p, x0 + kTW, y, k) : T(0);
        __syncthreads();
#pragma unroll
        for (int v = 0; v < kVX; ++v) {
            const int x = x0 + tx + kTX * v;
            if (yin && x < bx) {
                const int sc = (ty + 1) * kSW + tx + kTX * v + 1;
                const double L = laplacian_exact((double)c[v], (double)sm[sc - 1], (double)sm[sc + 1],
                                                 (double)sm[sc - kSW], (double)sm[sc + kSW], (double)zm[v],
                                                 (double)zp[v]);
                acc = fma(L, L, acc);
            }
            zm[v] = c[v];
            c[v] = zp[v];
        }
        __syncthreads();
    }
    const int tid = ty * kTX + tx;
    red[tid] = acc;
    __syncthreads();
    for (int s = kTX * kTY / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    if (tid == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* partials, int n, double* out)
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

// Face f of block d: the cells of the plane, first axis fastest.
__device__ __forceinline__ int face_size(const BlockDesc& d, int f)
{
    const int a = f >> 1;  // 0: x face (by x bz), 1: y face (bx x bz), 2: z face (bx x by)
    return a == 0 ? d.ext[1] * d.ext[2] : (a == 1 ? d.ext[0] * d.ext[2] : d.ext[0] * d.ext[1]);
}

// q-th cell of face f; `layer` = 0 selects the outermost interior plane
// (what is packed), 1 the ghost plane beyond it (where it is unpacked).
__device__ __forceinline__ void face_cell(const BlockDesc& d, int f, int q, int ghost, int& x, int& y, int& k)
{
    const int a = f >> 1, hi = f & 1;
    if (a == 0) {
        y = q % d.ext[1];
        k = q / d.ext[1];
        x = hi ? (ghost ? d.ext[0] : d.ext[0] - 1) : (ghost ? -1 : 0);
    } else if (a == 1) {
        x = q % d.ext[0];
        k = q / d.ext[0];
        y = hi ? (ghost ? d.ext[1] : d.ext[1] - 1) : (ghost ? -1 : 0);
    } else {
        x = q % d.ext[0];
        y = q / d.ext[0];
        k = hi ? (ghost ? d.ext[2] : d.ext[2] - 1) : (ghost ? -1 : 0);
    }
}

template <typename T>
__global__ void k_pack_face(const T* pool, const BlockDesc* desc, int b, int f, int p, T* send)
{
    const BlockDesc& d = desc[b];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= face_size(d, f)) return;
    int x, y, k;
    face_cell(d, f, q, 0, x, y, k);
    send[q] = pool[cell_index<T>(d, p, x, y, k)];
}

template <typename T>
__global__ void k_unpack_face(T* pool, const BlockDesc* desc, int b, int f, int p, const T* recv)
{
    const BlockDesc& d = desc[b];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= face_size(d, f)) return;
    int x, y, k;
    face_cell(d, f, q, 1, x, y, k);
    pool[cell_index<T>(d, p, x, y, k)] = recv[q];
}

// Six faces in one launch, one thread per cell of the largest face; faces at
// the global boundary are skipped. `faceoff` gives each face's offset in the
// block's halo segment.
template <typename T>
__global__ void k_pack6(const T* pool, const BlockDesc* desc, int b, int p, T* send, const int64_t* faceoff)
{
    const BlockDesc& d = desc[b];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
        if (d.nbr[f] < 0 || q >= face_size(d, f)) continue;
        int x, y, k;
        face_cell(d, f, q, 0, x, y, k);
        send[faceoff[f] + q] = pool[cell_index<T>(d, p, x, y, k)];
    }
}

template <typename T>
__global__ void k_unpack6(T* pool, const BlockDesc* desc, int b, int p, const T* recv, const int64_t* faceoff)
{
    const BlockDesc& d = desc[b];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
        if (d.nbr[f] < 0 || q >= face_size(d, f)) continue;
        int x, y, k;
        face_cell(d, f, q, 1, x, y, k);
        pool[cell_index<T>(d, p, x, y, k)] = recv[faceoff[f] + q];
    }
}

// Dense x-fastest instance arrays <-> block interiors (buffer p). Grid x is
// the block, grid y strides over the block's rows; threads walk x.
template <typename TS, typename TD>
__global__ void k_scatter(const TS* dense, TD* pool, const BlockDesc* desc, int p)
{
    const BlockDesc& d = desc[blockIdx.x];
    const int rows = d.ext[1] * d.ext[2];
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = r % d.ext[1], k = r / d.ext[1];
        const int64_t g = d.dense + (int64_t)d.org[0] +
                          (int64_t)d.gdim[0] * ((int64_t)(d.org[1] + y) + (int64_t)d.gdim[1] * (d.org[2] + k));
        for (int x = threadIdx.x; x < d.ext[0]; x += blockDim.x)
            pool[cell_index<TD>(d, p, x, y, k)] = (TD)dense[g + x];
    }
}

template <typename TS, typename TD>
__global__ void k_gather(const TS* pool, TD* dense, const BlockDesc* desc, int p)
{
    const BlockDesc& d = desc[blockIdx.x];
    const int rows = d.ext[1] * d.ext[2];
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = r % d.ext[1], k = r / d.ext[1];
        const int64_t g = d.dense + (int64_t)d.org[0] +
                          (int64_t)d.gdim[0] * ((int64_t)(d.org[1] + y) + (int64_t)d.gdim[1] * (d.org[2] + k));
        for (int x = threadIdx.x; x < d.ext[0]; x += blockDim.x)
            dense[g + x] = (TD)pool[cell_index<TS>(d, p, x, y, k)];
    }
}

// Dirichlet values into the ghost planes of faces at the global boundary,
// both buffers. One CTA per (block, face).
template <typename T>
__global__ void k_init_ghosts(T* pool, const BlockDesc* desc)
{
    const BlockDesc& d = desc[blockIdx.x];
    const int f = blockIdx.y;
    if (d.nbr[f] >= 0) return;
    const int n = face_size(d, f);
    const T v = (T)d.bc[f];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        int x, y, k;
        face_cell(d, f, q, 1, x, y, k);
        pool[cell_index<T>(d, 0, x, y, k)] = v;
        pool[cell_index<T>(d, 1, x, y, k)] = v;
    }
}

// ---------------------------------------------------------------- launchers

static inline dim3 tile_block() { return dim3(kTX, kTY, 1); }

int tile_width() { return kTW; }
int tile_height() { return kTY; }

template <typename T>
static cudaError_t stencil_block_t(const LaunchArgs& a, int arith, int b, int nx_tiles, int ny_tiles, int p,
                                   cudaStream_t s)
{
    dim3 grid(nx_tiles, ny_tiles, 1);
    if (sizeof(T) == 8 && arith == 1)
        k_stencil_block<T, 1><<<grid, tile_block(), 0, s>>>((T*)a.pool, a.desc, b, p);
    else
        k_stencil_block<T, 0><<<grid, tile_block(), 0, s>>>((T*)a.pool, a.desc, b, p);
    return cudaGetLastError();
}

cudaError_t launch_stencil_block(const LaunchArgs& a, int dtype_f32, int arith, int b, int nx_tiles, int ny_tiles,
                                 int p, cudaStream_t s)
{
    return dtype_f32 ? stencil_block_t<float>(a, arith, b, nx_tiles, ny_tiles, p, s)
                     : stencil_block_t<double>(a, arith, b, nx_tiles, ny_tiles, p, s);
}

template <typename T>
static cudaError_t fused_step_t(const LaunchArgs& a, int arith, int p, cudaStream_t s)
{
    if (sizeof(T) == 8 && arith == 1)
        k_fused_step<T, 1><<<a.nunits, tile_block(), 0, s>>>((T*)a.pool, a.desc, a.units, p);
    else
        k_fused_step<T, 0><<<a.nunits, tile_block(), 0, s>>>((T*)a.pool, a.desc, a.units, p);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const LaunchArgs& a, int dtype_f32, int arith, int p, cudaStream_t s)
{
    return dtype_f32 ? fused_step_t<float>(a, arith, p, s) : fused_step_t<double>(a, arith, p, s);
}

template <typename T, int ARITH>
static const void* persistent_fn()
{
    return (const void*)k_persistent<T, ARITH>;
}

const void* persistent_kernel(int dtype_f32, int arith)
{
    if (dtype_f32) return persistent_fn<float, 0>();
    return arith == 1 ? persistent_fn<double, 1>() : persistent_fn<double, 0>();
}

int persistent_block_threads() { return kTX * kTY; }

template <typename T>
static cudaError_t persistent_t(const LaunchArgs& a, const PersistentArgs& q, int arith, int ctas, cudaStream_t s)
{
    if (sizeof(T) == 8 && arith == 1)
        k_persistent<T, 1><<<ctas, tile_block(), 0, s>>>((T*)a.pool, a.desc, a.units, a.nunits, q.p0, q.n_iters,
                                                         q.done, q.work, q.status, q.wait_ns, q.hold_block,
                                                         q.hold_after);
    else
        k_persistent<T, 0><<<ctas, tile_block(), 0, s>>>((T*)a.pool, a.desc, a.units, a.nunits, q.p0, q.n_iters,
                                                         q.done, q.work, q.status, q.wait_ns, q.hold_block,
                                                         q.hold_after);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const LaunchArgs& a, const PersistentArgs& q, int dtype_f32, int arith, int ctas,
                              cudaStream_t s)
{
    return dtype_f32 ? persistent_t<float>(a, q, arith, ctas, s) : persistent_t<double>(a, q, arith, ctas, s);
}

cudaError_t launch_residual(const LaunchArgs& a, int dtype_f32, int p, double* partials, double* out,
                            cudaStream_t s)
{
    if (dtype_f32)
        k_residual<float><<<a.nunits, tile_block(), 0, s>>>((const float*)a.pool, a.desc, a.units, p, partials);
    else
        k_residual<double><<<a.nunits, tile_block(), 0, s>>>((const double*)a.pool, a.desc, a.units, p, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, s>>>(partials, a.nunits, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_face(const LaunchArgs& a, int dtype_f32, int b, int f, int p, void* send, int n,
                             cudaStream_t s)
{
    const int th = 128, g = (n + th - 1) / th;
    if (dtype_f32) k_pack_face<float><<<g, th, 0, s>>>((const float*)a.pool, a.desc, b, f, p, (float*)send);
    else k_pack_face<double><<<g, th, 0, s>>>((const double*)a.pool, a.desc, b, f, p, (double*)send);
    return cudaGetLastError();
}

cudaError_t launch_unpack_face(const LaunchArgs& a, int dtype_f32, int b, int f, int p, const void* recv, int n,
                               cudaStream_t s)
{
    const int th = 128, g = (n + th - 1) / th;
    if (dtype_f32) k_unpack_face<float><<<g, th, 0, s>>>((float*)a.pool, a.desc, b, f, p, (const float*)recv);
    else k_unpack_face<double><<<g, th, 0, s>>>((double*)a.pool, a.desc, b, f, p, (const double*)recv);
    return cudaGetLastError();
}

cudaError_t launch_pack6(const LaunchArgs& a, int dtype_f32, int b, int p, void* send, const int64_t* faceoff,
                         int maxface, cudaStream_t s)
{
    const int th = 128, g = (maxface + th - 1) / th;
    if (dtype_f32) k_pack6<float><<<g, th, 0, s>>>((const float*)a.pool, a.desc, b, p, (float*)send, faceoff);
    else k_pack6<double><<<g, th, 0, s>>>((const double*)a.pool, a.desc, b, p, (double*)send, faceoff);
    return cudaGetLastError();
}

cudaError_t launch_unpack6(const LaunchArgs& a, int dtype_f32, int b, int p, const void* recv, const int64_t* faceoff,
                           int maxface, cudaStream_t s)
{
    const int th = 128, g = (maxface + th - 1) / th;
    if (dtype_f32) k_unpack6<float><<<g, th, 0, s>>>((float*)a.pool, a.desc, b, p, (const float*)recv, faceoff);
    else k_unpack6<double><<<g, th, 0, s>>>((double*)a.pool, a.desc, b, p, (const double*)recv, faceoff);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const LaunchArgs& a, int dtype_f32, int src_f32, const void* dense, int p, cudaStream_t s)
{
    dim3 grid(a.nblocks, 16, 1);
    if (dtype_f32) {
        if (src_f32) k_scatter<float, float><<<grid, 256, 0, s>>>((const float*)dense, (float*)a.pool, a.desc, p);
        else k_scatter<double, float><<<grid, 256, 0, s>>>((const double*)dense, (float*)a.pool, a.desc, p);
    } else {
        k_scatter<double, double><<<grid, 256, 0, s>>>((const double*)dense, (double*)a.pool, a.desc, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const LaunchArgs& a, int dtype_f32, int dst_f32, void* dense, int p, cudaStream_t s)
{
    dim3 grid(a.nblocks, 16, 1);
    if (dtype_f32) {
        if (dst_f32) k_gather<float, float><<<grid, 256, 0, s>>>((const float*)a.pool, (float*)dense, a.desc, p);
        else k_gather<float, double><<<grid, 256, 0, s>>>((const float*)a.pool, (double*)dense, a.desc, p);
    } else {
        k_gather<double, double><<<grid, 256, 0, s>>>((const double*)a.pool, (double*)dense, a.desc, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_ghosts(const LaunchArgs& a, int dtype_f32, cudaStream_t s)
{
    dim3 grid(a.nblocks, 6, 1);
    if (dtype_f32) k_init_ghosts<float><<<grid, 256, 0, s>>>((float*)a.pool, a.desc);
    else k_init_ghosts<double><<<grid, 256, 0, s>>>((double*)a.pool, a.desc);
    return cudaGetLastError();
}

}  // namespace jac
