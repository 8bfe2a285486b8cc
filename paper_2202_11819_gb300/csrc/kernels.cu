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
#include <type_traits>

#include "arith.cuh"
#include "jac_common.cuh"
#include "launch.h"

namespace jac {

// Tile of the z-marching update: 512 threads, one column each, as TW x
// (512 / TW) columns of a block; TW (16, 32 or 64) is chosen per context (the
// autotuner times the three). Each tile covers a z range [z0, z1) of the
// block, so the z depth of a work unit is chosen too.
constexpr int kThreads = 512;

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

template <typename T, int UNUSED>
__device__ __forceinline__ T mean7(T c, T xm, T xp, T ym, T yp, T zm, T zp)
{
    if constexpr (sizeof(T) == 4) return mean7_seq_f32(c, xm, xp, ym, yp, zm, zp);
    else return mean7_seq(c, xm, xp, ym, yp, zm, zp);
}

constexpr int OP_SEQ = 0;    // binary64/binary32 left-to-right sum / 7 in floating point
constexpr int OP_EXACT = 1;  // binary64 correctly rounded mean, grid-frame integer arithmetic
constexpr int OP_RES = 2;    // residual: sum of L^2 with the exact Laplacian term

template <typename T, int OP>
struct Elem {
    using type = frame::W96;
};
template <typename T>
struct Elem<T, OP_SEQ> {
    using type = T;
};

template <typename T>
__device__ __forceinline__ const T* bc_ptr(const BlockDesc& d, int f);
template <>
__device__ __forceinline__ const double* bc_ptr<double>(const BlockDesc& d, int f)
{
    return &d.bc[f];
}
template <>
__device__ __forceinline__ const float* bc_ptr<float>(const BlockDesc& d, int f)
{
    return &d.bcf[f];
}

template <typename T, bool CG>
__device__ __forceinline__ T ldv(const T* p)
{
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

template <typename T, int OP>
__device__ __forceinline__ typename Elem<T, OP>::type conv(T v, int eref)
{
    if constexpr (OP == OP_SEQ) return v;
    else return frame::of((double)v, eref);
}

// Where the value of (x, y) lives along z, for -1 <= x <= bx, -1 <= y <= by
// with at most one coordinate outside the block: plane k is p[k * stride].
// PULL: outside cells come from the neighbouring block (stride: its plane) or
// are the Dirichlet constant (stride 0). Otherwise the block's ghost layer.
template <typename T>
struct Src {
    const T* p;
    int64_t stride;
};

template <typename T, bool PULL>
__device__ __forceinline__ Src<T> xy_source(const T* pool, const BlockDesc* desc, const BlockDesc& d, int p, int x,
                                            int y)
{
    if constexpr (PULL) {
        int f = -1;
        if (x < 0) f = 0;
        else if (x >= d.ext[0]) f = 1;
        else if (y < 0) f = 2;
        else if (y >= d.ext[1]) f = 3;
        if (f >= 0) {
            const int nb = d.nbr[f];
            if (nb < 0) return {bc_ptr<T>(d, f), 0};
            const BlockDesc& n = desc[nb];
            const int xx = f == 0 ? n.ext[0] - 1 : (f == 1 ? 0 : x);
            const int yy = f == 2 ? n.ext[1] - 1 : (f == 3 ? 0 : y);
            return {pool + cell_index<T>(n, p, xx, yy, 0), n.plane};
        }
    }
    return {pool + cell_index<T>(d, p, x, y, 0), d.plane};
}

// The value of column (x, y) at plane -1 (zface 4) or plane bz (zface 5).
template <typename T, bool PULL>
__device__ __forceinline__ const T* z_source(const T* pool, const BlockDesc* desc, const BlockDesc& d, int p, int x,
                                             int y, int zface)
{
    if constexpr (PULL) {
        const int nb = d.nbr[zface];
        if (nb < 0) return bc_ptr<T>(d, zface);
        const BlockDesc& n = desc[nb];
        return pool + cell_index<T>(n, p, x, y, zface == 4 ? n.ext[2] - 1 : 0);
    }
    return pool + cell_index<T>(d, p, x, y, zface == 4 ? -1 : d.ext[2]);
}

// Exact per-cell path for the rare cells the grid frame cannot hold: the
// seven raw values are re-read and handed to the per-cell exact routines.
template <typename T, bool PULL, bool CG, bool LAPLACIAN>
__device__ __noinline__ double exact_cell(const T* pool, const BlockDesc* desc, int b, int p, int x, int y, int k)
{
    const BlockDesc& d = desc[b];
    const double c = (double)ld<T, CG>(pool + cell_index<T>(d, p, x, y, k));
    const double xm = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x - 1, y, k);
    const double xp = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x + 1, y, k);
    const double ym = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x, y - 1, k);
    const double yp = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x, y + 1, k);
    const double zm = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x, y, k - 1);
    const double zp = (double)load_cell<T, PULL, CG>(pool, desc, d, p, x, y, k + 1);
    if constexpr (LAPLACIAN) return laplacian_exact(c, xm, xp, ym, yp, zm, zp);
    else return mean7_exact(c, xm, xp, ym, yp, zm, zp);
}

// Cells the grid frame cannot hold are not computed inside the z loop (a call
// there would make the compiler save registers on every plane); they are
// recorded here and recomputed with the exact per-cell routines once the
// tile's loop has finished. That is safe: until this tile reports completion
// neither its input buffer region nor its neighbours' faces can change.
constexpr int kSlowMax = 256;

struct SlowList {
    int n;
    uint32_t cell[kSlowMax];  // (k << 9) | tid
};

// The z-marching engine over one tile (x0 .. x0+TW-1, y0 .. y0+512/TW-1,
// planes z0 .. z1-1) of block b, reading buffer p.
//   OP_SEQ / OP_EXACT: writes the interior of buffer p^1;
//   OP_RES:           returns this thread's sum of L^2 (thread 0 also adds the
//                     cells recomputed exactly, in (k, tid) order).
// Every shared slot of the tile plane (the interior plus its halo ring) is a
// stream along z (pointer + plane stride, or a constant): own columns, halo
// cells that fall inside the tile where it overhangs the block edge, and one
// extra ring slot for each of the first 2 (TW + 512/TW) threads. Values are
// loaded D planes ahead into registers, converted once (to the grid frame for
// the exact ops), stored in a double-buffered shared plane (one barrier per
// plane), and the z neighbours are carried in registers.
template <typename T, int OP, bool PULL, bool CG, int D, int TW>
__device__ double tile_engine(T* __restrict__ pool, const BlockDesc* __restrict__ desc,
                              const int32_t* __restrict__ frame_e, int b, int p, int x0, int y0, int z0, int z1,
                              typename Elem<T, OP>::type* sm, SlowList* slow)
{
    using E = typename Elem<T, OP>::type;
    constexpr int kTX = TW, kTY = kThreads / TW, kTW = TW, kSW = TW + 2;
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int eref = (OP == OP_SEQ) ? 0 : frame_e[d.inst] + 1;
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const int x = x0 + tx, y = y0 + ty;
    const int64_t plane = d.plane;
    if (OP != OP_SEQ && tid == 0) slow->n = 0;

    // own column: 0 unused, 1 interior cell, 2 halo cell inside the tile
    int kind = 0;
    const T* sp = pool;
    int64_t ss = 0;
    const T* zhi = pool;  // the value above the last plane of the range
    int64_t oidx = 0;
    E wzm{}, wc{};
    T ring[D + 1];  // interior: planes k+1 .. k+1+D; halo: planes k .. k+D
#pragma unroll
    for (int i = 0; i <= D; ++i) ring[i] = T(0);
    if (x < bx && y < by) {
        kind = 1;
        sp = pool + cell_index<T>(d, p, x, y, 0);
        ss = plane;
        zhi = z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : sp + z1 * plane;
        oidx = cell_index<T>(d, p ^ 1, x, y, 0);
        const T* zlo = z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : sp + (z0 - 1) * plane;
        wzm = conv<T, OP>(ldv<T, CG>(zlo), eref);
        wc = conv<T, OP>(ldv<T, CG>(sp + z0 * plane), eref);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int q = z0 + 1 + i;
            ring[i] = q < z1 ? ldv<T, CG>(sp + q * ss) : (q == z1 ? ldv<T, CG>(zhi) : T(0));
        }
    } else if ((x == bx && y < by) || (y == by && x < bx)) {
        kind = 2;
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, x, y);
        sp = s.p;
        ss = s.stride;
#pragma unroll
        for (int i = 0; i < D; ++i) ring[i] = z0 + i < z1 ? ldv<T, CG>(sp + (z0 + i) * ss) : T(0);
    }
    // one ring slot per thread for tid < 2 (TW + TY): row y0-1, row y0+TY,
    // column x0-1, column x0+TW (only the slots some interior cell reads)
    int er = -1, ec = 0;
    const T* ep = pool;
    int64_t es = 0;
    T ering[D + 1];  // planes k .. k+D
#pragma unroll
    for (int i = 0; i <= D; ++i) ering[i] = T(0);
    if (tid < 2 * kTW + 2 * kTY) {
        int hx, hy;
        if (tid < kTW) {
            er = 0;
            ec = tid + 1;
            hx = x0 + tid;
            hy = y0 - 1;
            if (hx >= bx) er = -1;
        } else if (tid < 2 * kTW) {
            const int c = tid - kTW;
            er = kTY + 1;
            ec = c + 1;
            hx = x0 + c;
            hy = y0 + kTY;
            if (hx >= bx || hy > by) er = -1;
        } else if (tid < 2 * kTW + kTY) {
            const int r = tid - 2 * kTW;
            er = r + 1;
            ec = 0;
            hx = x0 - 1;
            hy = y0 + r;
            if (hy >= by) er = -1;
        } else {
            const int r = tid - 2 * kTW - kTY;
            er = r + 1;
            ec = kTW + 1;
            hx = x0 + kTW;
            hy = y0 + r;
            if (hy >= by || hx > bx) er = -1;
        }
        if (er >= 0) {
            const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, hx, hy);
            ep = s.p;
            es = s.stride;
#pragma unroll
            for (int i = 0; i < D; ++i) ering[i] = z0 + i < z1 ? ldv<T, CG>(ep + (z0 + i) * es) : T(0);
        }
    }
    if (OP != OP_SEQ) __syncthreads();  // slow->n = 0 visible before any append

    double acc = 0.0;
#pragma unroll 2
    for (int k = z0; k < z1; ++k) {
        E* buf = sm + (k & 1) * ((kTY + 2) * kSW);
        // issue the loads D planes ahead
        if (kind == 1) {
            const int q = k + 1 + D;
            ring[D] = q < z1 ? ldv<T, CG>(sp + q * ss) : (q == z1 ? ldv<T, CG>(zhi) : T(0));
        } else if (kind == 2) {
            ring[D] = k + D < z1 ? ldv<T, CG>(sp + (k + D) * ss) : T(0);
        }
        if (er >= 0) ering[D] = k + D < z1 ? ldv<T, CG>(ep + (k + D) * es) : T(0);
        // this plane's shared slots
        E* slot = buf + (ty + 1) * kSW + tx + 1;
        if (kind == 1) *slot = wc;
        else if (kind == 2) *slot = conv<T, OP>(ring[0], eref);
        if (er >= 0) buf[er * kSW + ec] = conv<T, OP>(ering[0], eref);
        __syncthreads();
        if (kind == 1) {
            const E wzp = conv<T, OP>(ring[0], eref);
            const int sc = (ty + 1) * kSW + tx + 1;
            if constexpr (OP == OP_SEQ) {
                pool[oidx + k * plane] = mean7<T, 0>(wc, buf[sc - 1], buf[sc + 1], buf[sc - kSW], buf[sc + kSW], wzm, wzp);
            } else {
                double o;
                bool ok;
                if constexpr (OP == OP_EXACT) {
                    ok = frame::mean7(wc, buf[sc - 1], buf[sc + 1], buf[sc - kSW], buf[sc + kSW], wzm, wzp, eref, o);
                    if (ok) pool[oidx + k * plane] = (T)o;
                } else {
                    ok = frame::laplacian(wc, buf[sc - 1], buf[sc + 1], buf[sc - kSW], buf[sc + kSW], wzm, wzp, eref, o);
                    if (ok) acc = fma(o, o, acc);
                }
                if (!ok) {
                    const int i = atomicAdd(&slow->n, 1);
                    if (i < kSlowMax) slow->cell[i] = ((uint32_t)k << 9) | (uint32_t)tid;
                }
            }
            wzm = wc;
            wc = wzp;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ring[i] = ring[i + 1];
            ering[i] = ering[i + 1];
        }
    }
    if constexpr (OP != OP_SEQ) {
        __syncthreads();
        const int n = slow->n;
        if (n > 0) {
            if (n <= kSlowMax) {
                if constexpr (OP == OP_EXACT) {
                    for (int i = tid; i < n; i += kThreads) {
                        const uint32_t c = slow->cell[i];
                        const int kk = (int)(c >> 9), t = (int)(c & 511u);
                        const int cx = x0 + t % kTX, cy = y0 + t / kTX;
                        pool[cell_index<T>(d, p ^ 1, cx, cy, kk)] =
                            (T)exact_cell<T, PULL, CG, false>(pool, desc, b, p, cx, cy, kk);
                    }
                } else if (tid == 0) {
                    // deterministic: ascending (k, tid)
                    for (int i = 1; i < n; ++i) {
                        const uint32_t v = slow->cell[i];
                        int j = i - 1;
                        while (j >= 0 && slow->cell[j] > v) {
                            slow->cell[j + 1] = slow->cell[j];
                            --j;
                        }
                        slow->cell[j + 1] = v;
                    }
                    for (int i = 0; i < n; ++i) {
                        const uint32_t c = slow->cell[i];
                        const int kk = (int)(c >> 9), t = (int)(c & 511u);
                        const double L = exact_cell<T, PULL, CG, true>(pool, desc, b, p, x0 + t % kTX, y0 + t / kTX, kk);
                        acc = fma(L, L, acc);
                    }
                }
            } else {
                // more cells outside the frame than the list holds: redo the
                // whole tile with the exact per-cell routines
                if constexpr (OP == OP_EXACT) {
                    if (kind == 1)
                        for (int kk = z0; kk < z1; ++kk)
                            pool[oidx + kk * plane] = (T)exact_cell<T, PULL, CG, false>(pool, desc, b, p, x, y, kk);
                } else {
                    acc = 0.0;
                    if (kind == 1)
                        for (int kk = z0; kk < z1; ++kk) {
                            const double L = exact_cell<T, PULL, CG, true>(pool, desc, b, p, x, y, kk);
                            acc = fma(L, L, acc);
                        }
                }
            }
        }
    }
    return acc;
}

template <typename T, int OP, int TW>
__host__ __device__ constexpr int smem_bytes()
{
    return 2 * (kThreads / TW + 2) * (TW + 2) * (int)sizeof(typename Elem<T, OP>::type);
}

// ---------------------------------------------------------------- lean engine
// For binary32 (the floating-point rule, cheap arithmetic) the
// arithmetic is cheap and the kernel must simply keep enough bytes in flight.
// Each thread owns one column of the tile and walks it along z with no
// shared memory and no barrier: its own values stream from DRAM DC planes
// ahead; its four x/y neighbours are read from short streams DN planes ahead,
// which hit L1 (their lines were requested DC - DN planes earlier by the
// neighbouring column's own stream); the z neighbours are carried in
// registers. Neighbours across a block face come from the neighbouring block
// (or are the Dirichlet constant, stride 0).
template <typename T>
constexpr int kLeanDC = 11;
constexpr int kLeanDN = 1;

template <typename T, bool PULL, bool CG, int TW>
__device__ __forceinline__ void lean_tile(T* __restrict__ pool, const BlockDesc* __restrict__ desc, int b, int p,
                                          int x0, int y0, int z0, int z1)
{
    constexpr int DC = kLeanDC<T>, DN = kLeanDN;
    const BlockDesc& d = desc[b];
    const int tid = threadIdx.x;
    const int x = x0 + tid % TW, y = y0 + tid / TW;
    if (x >= d.ext[0] || y >= d.ext[1]) return;
    const int bz = d.ext[2];
    const int64_t plane = d.plane;
    const T* pc = pool + cell_index<T>(d, p, x, y, 0);
    const int32_t plane32 = (int32_t)plane;
    const Src<T> s0 = xy_source<T, PULL>(pool, desc, d, p, x - 1, y);
    const Src<T> s1 = xy_source<T, PULL>(pool, desc, d, p, x + 1, y);
    const Src<T> s2 = xy_source<T, PULL>(pool, desc, d, p, x, y - 1);
    const Src<T> s3 = xy_source<T, PULL>(pool, desc, d, p, x, y + 1);
    // plane strides fit 32 bits (at most (256 + 2) x 512 elements)
    struct {
        const T* p;
        int32_t stride;
    } sxm{s0.p, (int32_t)s0.stride}, sxp{s1.p, (int32_t)s1.stride}, sym{s2.p, (int32_t)s2.stride},
        syp{s3.p, (int32_t)s3.stride};
    const T* zhi = z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : pc + z1 * plane;
    const T* zlo = z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : pc + (z0 - 1) * plane;
    T* out = pool + cell_index<T>(d, p ^ 1, x, y, 0);
    // Ring slots are fixed registers: the z loop is unrolled by the ring length
    // R so every slot index is a compile-time constant (moving a register whose
    // load is still in flight would wait for that load and undo the prefetch).
    // Own column: plane q sits in slot (q - z0 - 1) % R; neighbours: plane q
    // in slot (q - z0) % RN, with RN dividing R. Every stream walks with a
    // running pointer; chunks whose loads all fall inside [z0, z1) run without
    // range checks.
    constexpr int R = DC + 1, RN = DN + 1;
    static_assert(R % RN == 0, "neighbour ring must divide the column ring");
    T rc[R], rxm[RN], rxp[RN], rym[RN], ryp[RN];
#pragma unroll
    for (int i = 0; i < DC; ++i) {
        const int q = z0 + 1 + i;
        rc[i] = q < z1 ? ld<T, CG>(pc + q * plane32) : (q == z1 ? ld<T, CG>(zhi) : T(0));
    }
    const T* po = pc + (z0 + 1 + DC) * plane32;  // own stream: plane k + 1 + DC
    const T* pxm = sxm.p + z0 * sxm.stride;       // neighbour streams: plane k + DN
    const T* pxp = sxp.p + z0 * sxp.stride;
    const T* pym = sym.p + z0 * sym.stride;
    const T* pyp = syp.p + z0 * syp.stride;
#pragma unroll
    for (int i = 0; i < DN; ++i) {
        const bool in = z0 + i < z1;
        rxm[i] = in ? ld<T, CG>(pxm) : T(0);
        rxp[i] = in ? ld<T, CG>(pxp) : T(0);
        rym[i] = in ? ld<T, CG>(pym) : T(0);
        ryp[i] = in ? ld<T, CG>(pyp) : T(0);
        pxm += sxm.stride;
        pxp += sxp.stride;
        pym += sym.stride;
        pyp += syp.stride;
    }
    T zm = ld<T, CG>(zlo);
    T c = ld<T, CG>(pc + z0 * plane32);
    T* po_out = out + z0 * plane32;
    auto step = [&](auto full, int j, int k) {
        constexpr bool FULL = decltype(full)::value;
        const int sn = (j + R - 1) % R, sl = (j + DN) % RN, su = j % RN;
        if (FULL) {
            rc[sn] = ld<T, CG>(po);
            rxm[sl] = ld<T, CG>(pxm);
            rxp[sl] = ld<T, CG>(pxp);
            rym[sl] = ld<T, CG>(pym);
            ryp[sl] = ld<T, CG>(pyp);
        } else {
            const int q = k + 1 + DC;
            rc[sn] = q < z1 ? ld<T, CG>(po) : (q == z1 ? ld<T, CG>(zhi) : T(0));
            if (k + DN < z1) {
                rxm[sl] = ld<T, CG>(pxm);
                rxp[sl] = ld<T, CG>(pxp);
                rym[sl] = ld<T, CG>(pym);
                ryp[sl] = ld<T, CG>(pyp);
            }
        }
        po += plane32;
        pxm += sxm.stride;
        pxp += sxp.stride;
        pym += sym.stride;
        pyp += syp.stride;
        const T zp = rc[j];
        *po_out = mean7<T, 0>(c, rxm[su], rxp[su], rym[su], ryp[su], zm, zp);
        po_out += plane32;
        zm = c;
        c = zp;
    };
    int kb = z0;
    // full chunks: the last own load of the chunk, plane kb + R + DC, is < z1
    for (; kb + R + DC < z1; kb += R) {
#pragma unroll
        for (int j = 0; j < R; ++j) step(std::true_type{}, j, kb + j);
    }
    for (; kb < z1; kb += R) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (kb + j < z1) step(std::false_type{}, j, kb + j);
    }
}

template <typename T, int TW>
__global__ void __launch_bounds__(kThreads, 2) k_fused_lean(T* pool, const BlockDesc* desc, const TileUnit* units, int p)
{
    const TileUnit u = units[blockIdx.x];
    lean_tile<T, true, false, TW>(pool, desc, u.block, p, u.x0, u.y0, u.z0, u.z1);
}

// prefetch depth: binary32 tiles are bandwidth-bound and need more bytes in
// flight; binary64 tiles are bound by the arithmetic
template <typename T>
constexpr int kDepth = sizeof(T) == 4 ? 6 : 3;

template <typename T, int OP, int TW>
__global__ void __launch_bounds__(kThreads, 2) k_stencil_block(T* pool, const BlockDesc* desc, const int32_t* frame_e,
                                                               int b, int p)
{
    __shared__ __align__(16) unsigned char sm[smem_bytes<T, OP, TW>()];
    __shared__ SlowList slow;
    tile_engine<T, OP, false, false, kDepth<T>, TW>(pool, desc, frame_e, b, p, blockIdx.x * TW,
                                                    blockIdx.y * (kThreads / TW), 0, desc[b].ext[2],
                                                    (typename Elem<T, OP>::type*)sm, &slow);
}

template <typename T, int OP, int TW>
__global__ void __launch_bounds__(kThreads, 2) k_fused_step(T* pool, const BlockDesc* desc, const int32_t* frame_e,
                                                            const TileUnit* units, int p)
{
    __shared__ __align__(16) unsigned char sm[smem_bytes<T, OP, TW>()];
    __shared__ SlowList slow;
    const TileUnit u = units[blockIdx.x];
    tile_engine<T, OP, true, false, kDepth<T>, TW>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1,
                                                   (typename Elem<T, OP>::type*)sm, &slow);
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
// overwrites (buffer p^1 held iteration t-1). The seven counters are polled
// by seven threads at once, and the next unit is taken while the current
// one computes. Every wait is bounded.
template <typename T, int OP, int TW, bool LEAN>
__global__ void __launch_bounds__(kThreads, 2)
    k_persistent(T* pool, const BlockDesc* desc, const int32_t* frame_e, const TileUnit* units, int nunits, int p0,
                 int64_t n_iters, uint32_t* done, unsigned long long* work, DeviceStatus* st, int64_t wait_ns,
                 int hold_block, int64_t hold_after)
{
    __shared__ __align__(16) unsigned char sm[smem_bytes<T, OP, TW>()];
    __shared__ SlowList slow;
    __shared__ long long s_next;
    __shared__ int s_stop;
    const long long total = (long long)n_iters * nunits;
    const int tid = threadIdx.x;
    if (tid == 0) s_next = (long long)atomicAdd(work, 1ull);
    __syncthreads();
    for (;;) {
        const long long w = s_next;
        if (w >= total) break;
        const int t = (int)(w / nunits);
        const TileUnit u = units[w % nunits];
        if (tid == 0) s_stop = 0;
        __syncthreads();
        if (t > 0 && tid < 7) {
            const int n = tid == 0 ? u.block : desc[u.block].nbr[tid - 1];
            if (n >= 0) {
                const uint32_t need = (uint32_t)t * (uint32_t)desc[n].ntiles;
                const uint64_t t0 = global_ns();
                unsigned ns = 32;
                while (ld_acquire(done + n) < need) {
                    if (ld_volatile(&st->abort)) {
                        s_stop = 1;
                        break;
                    }
                    if ((int64_t)(global_ns() - t0) > wait_ns) {
                        if (atomicCAS(&st->err, kErrNone, kErrTimeout) == kErrNone) {
                            st->where_block = n;
                            st->where_iter = t;
                        }
                        atomicExch(&st->abort, 1);
                        s_stop = 1;
                        break;
                    }
                    __nanosleep(ns);
                    ns = ns < 1024 ? ns * 2 : ns;
                }
                __threadfence();
            }
        }
        __syncthreads();
        if (s_stop) break;
        // take the next unit now; its index is read after this one finishes
        if (tid == 0) s_next = ld_volatile(&st->abort) ? total : (long long)atomicAdd(work, 1ull);
        if constexpr (LEAN) {
            // plain (L1-cached) loads are safe here: the acquire and the
            // barrier above order them after the neighbours' releases
            lean_tile<T, true, false, TW>(pool, desc, u.block, (p0 + t) & 1, u.x0, u.y0, u.z0, u.z1);
        } else {
            tile_engine<T, OP, true, true, kDepth<T>, TW>(pool, desc, frame_e, u.block, (p0 + t) & 1, u.x0, u.y0,
                                                          u.z0, u.z1, (typename Elem<T, OP>::type*)sm, &slow);
        }
        __syncthreads();
        if (tid == 0 && !(u.block == hold_block && t >= hold_after)) {
            __threadfence();
            atomicAdd(done + u.block, 1u);
        }
    }
}

// Residual: per CTA the sum over its tile of L^2 (L the exact Laplacian term
// rounded once), in a fixed order (per thread over k, then a fixed tree).
template <typename T, int TW>
__global__ void __launch_bounds__(kThreads, 2) k_residual(const T* pool, const BlockDesc* desc,
                                                          const int32_t* frame_e, const TileUnit* units, int p,
                                                          double* partials)
{
    __shared__ __align__(16) unsigned char sm[smem_bytes<T, OP_RES, TW>()];
    __shared__ SlowList slow;
    __shared__ double red[kThreads];
    const TileUnit u = units[blockIdx.x];
    const double acc = tile_engine<T, OP_RES, true, false, 2, TW>(const_cast<T*>(pool), desc, frame_e, u.block, p,
                                                                  u.x0, u.y0, u.z0, u.z1, (frame::W96*)sm, &slow);
    const int tid = threadIdx.x;
    red[tid] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    if (tid == 0) partials[blockIdx.x] = red[0];
}

// Per-grid residuals: resident grid i (slot slot[i]) owns partials
// [seg[i], seg[i+1]); one CTA per grid sums them in a fixed order.
__global__ void k_sum_segments(const double* partials, const int32_t* seg, const int32_t* slot, double* out)
{
    __shared__ double red[256];
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int j = seg[i] + (int)threadIdx.x; j < seg[i + 1]; j += blockDim.x) acc = acc + partials[j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[slot[i]] = sqrt(red[0]);
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
__global__ void k_scatter(const TS* dense, TD* pool, const BlockDesc* desc, int b0, int64_t dense_base, int p,
                          int32_t* frame_e)
{
    const BlockDesc& d = desc[b0 + blockIdx.x];
    const int rows = d.ext[1] * d.ext[2];
    int emax = 0;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = r % d.ext[1], k = r / d.ext[1];
        const int64_t g = d.dense - dense_base + (int64_t)d.org[0] +
                          (int64_t)d.gdim[0] * ((int64_t)(d.org[1] + y) + (int64_t)d.gdim[1] * (d.org[2] + k));
        for (int x = threadIdx.x; x < d.ext[0]; x += blockDim.x) {
            const TD v = (TD)dense[g + x];
            pool[cell_index<TD>(d, p, x, y, k)] = v;
            emax = max(emax, (int)((dbits((double)v) >> 52) & 0x7FF));
        }
    }
    // largest exponent field of the instance: the grid frame's reference
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(frame_e + d.inst, emax);
}

template <typename TS, typename TD>
__global__ void k_gather(const TS* pool, TD* dense, const BlockDesc* desc, int b0, int64_t dense_base, int p)
{
    const BlockDesc& d = desc[b0 + blockIdx.x];
    const int rows = d.ext[1] * d.ext[2];
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = r % d.ext[1], k = r / d.ext[1];
        const int64_t g = d.dense + (int64_t)d.org[0] +
                          (int64_t)d.gdim[0] * ((int64_t)(d.org[1] + y) + (int64_t)d.gdim[1] * (d.org[2] + k));
        for (int x = threadIdx.x; x < d.ext[0]; x += blockDim.x)
            dense[g - dense_base + x] = (TD)pool[cell_index<TS>(d, p, x, y, k)];
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

int tile_rows(int tw) { return kThreads / tw; }
int engine_threads() { return kThreads; }
bool tile_width_supported(int tw) { return tw == 16 || tw == 32 || tw == 64; }

#define JAC_TW_DISPATCH(tw, CALL) \
    switch (tw) {                 \
        case 16: {                \
            constexpr int TW = 16; \
            CALL;                 \
            break;                \
        }                         \
        case 64: {                \
            constexpr int TW = 64; \
            CALL;                 \
            break;                \
        }                         \
        default: {                \
            constexpr int TW = 32; \
            CALL;                 \
            break;                \
        }                         \
    }

template <typename T, int TW>
static void stencil_block_t(const LaunchArgs& a, int arith, int b, int nx_tiles, int ny_tiles, int p, cudaStream_t s)
{
    dim3 grid(nx_tiles, ny_tiles, 1);
    if constexpr (sizeof(T) == 8) {
        if (arith == 1) {
            k_stencil_block<T, OP_EXACT, TW><<<grid, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, b, p);
            return;
        }
    }
    k_stencil_block<T, OP_SEQ, TW><<<grid, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, b, p);
}

cudaError_t launch_stencil_block(const LaunchArgs& a, int dtype_f32, int arith, int b, int nx_tiles, int ny_tiles,
                                 int p, cudaStream_t s)
{
    if (dtype_f32) JAC_TW_DISPATCH(a.tile_w, (stencil_block_t<float, TW>(a, arith, b, nx_tiles, ny_tiles, p, s)))
    else JAC_TW_DISPATCH(a.tile_w, (stencil_block_t<double, TW>(a, arith, b, nx_tiles, ny_tiles, p, s)))
    return cudaGetLastError();
}

template <typename T, int TW>
static void fused_step_t(const LaunchArgs& a, int arith, int p, cudaStream_t s)
{
    if constexpr (sizeof(T) == 8) {
        if (arith == 1) {
            k_fused_step<T, OP_EXACT, TW><<<a.nunits, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, a.units, p);
            return;
        }
    }
    if constexpr (sizeof(T) == 4)
        k_fused_lean<T, TW><<<a.nunits, kThreads, 0, s>>>((T*)a.pool, a.desc, a.units, p);
    else
        k_fused_step<T, OP_SEQ, TW><<<a.nunits, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, a.units, p);
}

cudaError_t launch_fused_step(const LaunchArgs& a, int dtype_f32, int arith, int p, cudaStream_t s)
{
    if (dtype_f32) JAC_TW_DISPATCH(a.tile_w, (fused_step_t<float, TW>(a, arith, p, s)))
    else JAC_TW_DISPATCH(a.tile_w, (fused_step_t<double, TW>(a, arith, p, s)))
    return cudaGetLastError();
}

template <int TW>
static const void* persistent_fn(int dtype_f32, int arith)
{
    if (dtype_f32) return (const void*)k_persistent<float, OP_SEQ, TW, true>;
    return arith == 1 ? (const void*)k_persistent<double, OP_EXACT, TW, false>
                      : (const void*)k_persistent<double, OP_SEQ, TW, false>;
}

const void* persistent_kernel(int dtype_f32, int arith, int tw)
{
    const void* f = nullptr;
    JAC_TW_DISPATCH(tw, (f = persistent_fn<TW>(dtype_f32, arith)))
    return f;
}

int persistent_block_threads() { return kThreads; }

template <typename T, int TW>
static void persistent_t(const LaunchArgs& a, const PersistentArgs& q, int arith, int ctas, cudaStream_t s)
{
    if constexpr (sizeof(T) == 8) {
        if (arith == 1) {
            k_persistent<T, OP_EXACT, TW, false><<<ctas, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, a.units, a.nunits,
                                                                    q.p0, q.n_iters, q.done, q.work, q.status,
                                                                    q.wait_ns, q.hold_block, q.hold_after);
            return;
        }
    }
    k_persistent<T, OP_SEQ, TW, sizeof(T) == 4><<<ctas, kThreads, 0, s>>>((T*)a.pool, a.desc, a.frame, a.units, a.nunits, q.p0,
                                                          q.n_iters, q.done, q.work, q.status, q.wait_ns,
                                                          q.hold_block, q.hold_after);
}

cudaError_t launch_persistent(const LaunchArgs& a, const PersistentArgs& q, int dtype_f32, int arith, int ctas,
                              cudaStream_t s)
{
    if (dtype_f32) JAC_TW_DISPATCH(a.tile_w, (persistent_t<float, TW>(a, q, arith, ctas, s)))
    else JAC_TW_DISPATCH(a.tile_w, (persistent_t<double, TW>(a, q, arith, ctas, s)))
    return cudaGetLastError();
}

cudaError_t launch_residual_partials(const LaunchArgs& a, int dtype_f32, int p, double* partials, cudaStream_t s)
{
    if (dtype_f32)
        JAC_TW_DISPATCH(a.tile_w, (k_residual<float, TW><<<a.nunits, kThreads, 0, s>>>(
                                      (const float*)a.pool, a.desc, a.frame, a.units, p, partials)))
    else
        JAC_TW_DISPATCH(a.tile_w, (k_residual<double, TW><<<a.nunits, kThreads, 0, s>>>(
                                      (const double*)a.pool, a.desc, a.frame, a.units, p, partials)))
    return cudaGetLastError();
}

cudaError_t launch_residual(const LaunchArgs& a, int dtype_f32, int p, double* partials, double* out,
                            cudaStream_t s)
{
    cudaError_t e = launch_residual_partials(a, dtype_f32, p, partials, s);
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, s>>>(partials, a.nunits, out);
    return cudaGetLastError();
}

cudaError_t launch_residual_segments(const LaunchArgs& a, int dtype_f32, int p, double* partials, const int32_t* seg,
                                     const int32_t* slot, int nseg, double* out, cudaStream_t s)
{
    cudaError_t e = launch_residual_partials(a, dtype_f32, p, partials, s);
    if (e != cudaSuccess) return e;
    k_sum_segments<<<nseg, 256, 0, s>>>(partials, seg, slot, out);
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

cudaError_t launch_scatter(const LaunchArgs& a, int dtype_f32, int src_f32, const void* dense, int b0, int nb,
                           int64_t dense_base, int p, cudaStream_t s)
{
    dim3 grid(nb, 16, 1);
    if (dtype_f32) {
        if (src_f32)
            k_scatter<float, float><<<grid, 256, 0, s>>>((const float*)dense, (float*)a.pool, a.desc, b0, dense_base,
                                                         p, a.frame);
        else
            k_scatter<double, float><<<grid, 256, 0, s>>>((const double*)dense, (float*)a.pool, a.desc, b0,
                                                          dense_base, p, a.frame);
    } else {
        k_scatter<double, double><<<grid, 256, 0, s>>>((const double*)dense, (double*)a.pool, a.desc, b0, dense_base,
                                                       p, a.frame);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const LaunchArgs& a, int dtype_f32, int dst_f32, void* dense, int b0, int nb,
                          int64_t dense_base, int p, cudaStream_t s)
{
    dim3 grid(nb, 16, 1);
    if (dtype_f32) {
        if (dst_f32)
            k_gather<float, float><<<grid, 256, 0, s>>>((const float*)a.pool, (float*)dense, a.desc, b0, dense_base, p);
        else
            k_gather<float, double><<<grid, 256, 0, s>>>((const float*)a.pool, (double*)dense, a.desc, b0, dense_base,
                                                         p);
    } else {
        k_gather<double, double><<<grid, 256, 0, s>>>((const double*)a.pool, (double*)dense, a.desc, b0, dense_base,
                                                      p);
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
