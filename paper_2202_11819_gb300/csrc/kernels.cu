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
//   k_fused_step / k_fused_ring   unpack + update + pack of every block in one
//                                 launch (strategy C): ghost values are read
//                                 straight from the neighbouring blocks
//                                 (k_fused_ring: binary32, whose update needs
//                                 no frame conversion),
//   k_persistent                  all blocks and all iterations in one launch,
//                                 each tile waiting only for the previous
//                                 iteration of its own and neighbouring blocks
//                                 (the device form of the per-iteration
//                                 reference numbers of Section II-A),
//   k_narrow_residual /           the residual norm (binary64 / binary32),
//   k_ring_residual               alone or inside an update iteration,
//                                 deterministic order,
//   k_scatter / k_gather          dense x-fastest arrays <-> block storage.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <utility>

#include "arith.cuh"
#include "jac_common.cuh"
#include "launch.h"

namespace jac {

// Tile of the z-marching update: 512 threads, one column each, as TW x
// (512 / TW) columns of a block; TW (16, 32 or 64) is chosen per context (the
// autotuner times the three). Each tile covers a z range [z0, z1) of the
// block, so the z depth of a work unit is chosen too.
constexpr int kThreads = 512;  // the most threads of any engine CTA (slow-list encoding)
// Threads per CTA of the engines: 256 for binary64 (the exact mean's integer
// work schedules better in smaller CTAs, four per SM), 512 for binary32 (two
// per SM). A binary32 work unit is 1024 / TW rows (two columns per thread).
template <typename T>
constexpr int kNT = sizeof(T) == 8 ? 256 : 512;
template <typename T>
constexpr int kMinCTAs = 1024 / kNT<T>;
static_assert(kNT<float> <= kThreads && kNT<double> <= kThreads, "the slow lists encode thread ids below kThreads");
// Minimum resident CTAs per SM of the update kernels (it sets their register
// budget). The exact mean's two-column engine keeps four cells' values live
// per thread: three 256-thread CTAs per SM at 80 registers, the 96-bit step
// without spills. The persistent kernel is also built for four CTAs at 64
// registers (1.8 KB of spill stores, in the 96-bit step), which grids with at
// least two waves of units take: there the fourth CTA hides the units'
// prologue latency (512^3, 64-wide tiles: 0.425 ms per iteration young and
// 0.447 aged against 0.436 and 0.451). Everywhere else three are faster: one
// block of 64^3 (0.039 against 0.052 ms), the fused form at 512^3 aged (0.509
// against 0.539), the batch of 256 small grids (1.89e11 against 1.66e11
// cell-updates/s).
template <typename T, int OP>
constexpr int kMinCTAsOp = (sizeof(T) == 8 && OP == 1) ? 3 : kMinCTAs<T>;
constexpr int kMinCTAsWide = 4;

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
constexpr int OP_RES32 = 3;  // the same for binary32 grids, L in a 64-bit frame and L^2 summed exactly

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

// The single-plane engine's double-buffered exchange plane (the sequential
// rule: the values themselves).
template <typename T, int OP, int TW>
__host__ __device__ constexpr int smem_bytes()
{
    static_assert(OP == OP_SEQ, "the single-plane engine runs the sequential rule");
    return 2 * (kNT<T> / TW + 2) * (TW + 2) * (int)sizeof(T);
}

// Extra ring slots of a tile (the halo ring around the TW x 512/TW interior).
template <typename T, int TW>
__host__ __device__ constexpr int ring_extra()
{
    static_assert(2 * TW + 2 * (kNT<T> / TW) <= kNT<T>, "every halo-ring slot needs a thread");
    return 2 * TW + 2 * (kNT<T> / TW);
}

// Shared memory of the engine: the double-buffered exchange plane, then the
// prefetch rings (RD planes of one value per thread, and RD planes of the halo
// ring slots), all in dynamic shared memory.
template <typename T, int OP, int TW, int RD>
__host__ __device__ constexpr int engine_bytes()
{
    return smem_bytes<T, OP, TW>() + RD * (kNT<T> + ring_extra<T, TW>()) * (int)sizeof(T);
}

// Planes in the per-stream rings: binary64 (whose exact arithmetic hides
// latency itself) keeps the ring short, since every byte of shared memory
// taken is L1 cache lost for the halo reads (6 planes measured faster than
// 8, 10 or 12); binary32 needs more in flight.
template <typename T>
constexpr int kRing = sizeof(T) == 8 ? 6 : 12;
constexpr int kRingRes = 6;

extern __shared__ __align__(16) unsigned char jac_dyn_sm[];

// Asynchronous global -> shared copies of one value (cp.async, cached in L1;
// completion is tracked per thread by commit / wait groups, so a thread that
// reads only its own copies needs no barrier).
template <int N>
__device__ __forceinline__ void cp_async(void* dst, const void* src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One halo-ring slot of the tile plane per thread for tid < 2 (TW + TY): row
// y0-1, row y0+TY, column x0-1, column x0+TW (only the slots some interior
// cell reads). er < 0: this thread has none; else (er, ec) is the slot in the
// shared plane and p + k * stride the value of plane k (z0 based).
template <typename T>
struct HaloSlot {
    int er, ec;
    const T* p;
    int64_t stride;
};

template <typename T, bool PULL, int TW>
__device__ __forceinline__ HaloSlot<T> halo_slot(const T* pool, const BlockDesc* desc, const BlockDesc& d, int p,
                                                 int x0, int y0, int z0, int tid)
{
    constexpr int kTW = TW, kTY = kNT<T> / TW;
    const int bx = d.ext[0], by = d.ext[1];
    HaloSlot<T> h{-1, 0, pool, 0};
    if (tid >= ring_extra<T, TW>()) return h;
    int hx, hy;
    if (tid < kTW) {
        h.er = 0;
        h.ec = tid + 1;
        hx = x0 + tid;
        hy = y0 - 1;
        if (hx >= bx) h.er = -1;
    } else if (tid < 2 * kTW) {
        const int c = tid - kTW;
        h.er = kTY + 1;
        h.ec = c + 1;
        hx = x0 + c;
        hy = y0 + kTY;
        if (hx >= bx || hy > by) h.er = -1;
    } else if (tid < 2 * kTW + kTY) {
        const int r = tid - 2 * kTW;
        h.er = r + 1;
        h.ec = 0;
        hx = x0 - 1;
        hy = y0 + r;
        if (hy >= by) h.er = -1;
    } else {
        const int r = tid - 2 * kTW - kTY;
        h.er = r + 1;
        h.ec = kTW + 1;
        hx = x0 + kTW;
        hy = y0 + r;
        if (hy >= by || hx > bx) h.er = -1;
    }
    if (h.er >= 0) {
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, hx, hy);
        h.p = s.p + z0 * s.stride;
        h.stride = s.stride;
    }
    return h;
}

// After a tile's z loop: recompute the cells recorded in the slow list (or
// the whole tile when the list overflowed) with the exact per-cell routines.
template <typename T, int OP, bool PULL, bool CG, int TW>
__device__ __forceinline__ double slow_cells(T* __restrict__ pool, const BlockDesc* __restrict__ desc,
                                             const BlockDesc& d, int b, int p, int x0, int y0, int z0, int z1,
                                             bool interior, int x, int y, int64_t oidx, double acc, SlowList* slow)
{
    constexpr int kTX = TW;
    const int tid = threadIdx.x;
    const int64_t plane = d.plane;
    if constexpr (OP != OP_SEQ) {
        __syncthreads();
        const int n = slow->n;
        if (n > 0) {
            if (n <= kSlowMax) {
                if constexpr (OP == OP_EXACT) {
                    for (int i = tid; i < n; i += kNT<T>) {
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
                    if (interior)
                        for (int kk = z0; kk < z1; ++kk)
                            pool[oidx + kk * plane] = (T)exact_cell<T, PULL, CG, false>(pool, desc, b, p, x, y, kk);
                } else {
                    acc = 0.0;
                    if (interior)
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

// The single-plane z-marching engine over one tile (x0 .. x0+TW-1, y0 ..
// y0+512/TW-1, planes z0 .. z1-1) of block b, reading buffer p and writing
// the interior of buffer p^1 by the sequential rule (the exact mean and the
// residuals run on the two-plane engine below).
// Every shared slot of the tile plane (the interior plus its halo ring) is a
// stream along z (pointer + plane stride, or a constant): own columns, halo
// cells that fall inside the tile where it overhangs the block edge, and one
// extra ring slot for each of the first 2 (TW + 512/TW) threads. Each stream
// is copied RD - 1 planes ahead into a per-thread ring in shared memory
// (cp.async: the data in flight holds no registers and the loop needs no
// register rotation); each value is stored in a double-buffered shared plane
// (one barrier per plane), and the z neighbours are carried in registers.
template <typename T, int OP, bool PULL, bool CG, int RD, int TW>
__device__ void tile_engine(T* __restrict__ pool, const BlockDesc* __restrict__ desc, int b, int p, int x0, int y0,
                            int z0, int z1, unsigned char* smraw)
{
    static_assert(OP == OP_SEQ, "the single-plane engine runs the sequential rule");
    using E = T;
    constexpr int kN = kNT<T>, kTX = TW, kTY = kN / TW, kSW = TW + 2, kEr = ring_extra<T, TW>();
    static_assert(RD >= 2, "ring depth");
    E* sm = (E*)smraw;
    T* rc = (T*)(smraw + smem_bytes<T, OP, TW>());  // [RD][kN]
    T* re = rc + RD * kN;                            // [RD][kEr]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const int x = x0 + tx, y = y0 + ty;
    const int64_t plane = d.plane;

    // own column: 0 unused, 1 interior cell, 2 halo cell inside the tile.
    // The value consumed at iteration k is at sp + (k - z0) * ss: kind 1 the
    // plane above (plane k + 1, and zhi for the last plane), kind 2 plane k.
    int kind = 0;
    const T* sp = pool;
    int64_t ss = 0;
    const T* zhi = pool;  // the value above the last plane of the range
    int64_t oidx = 0;
    E wzm{}, wc{};
    if (x < bx && y < by) {
        kind = 1;
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        ss = plane;
        sp = col + (z0 + 1) * plane;
        zhi = z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : col + z1 * plane;
        oidx = cell_index<T>(d, p ^ 1, x, y, 0);
        const T* zlo = z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : col + (z0 - 1) * plane;
        wzm = ldv<T, CG>(zlo);
        wc = ldv<T, CG>(col + z0 * plane);
    } else if ((x == bx && y < by) || (y == by && x < bx)) {
        kind = 2;
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, x, y);
        sp = s.p + z0 * s.stride;
        ss = s.stride;
    }
    const HaloSlot<T> hs = halo_slot<T, PULL, TW>(pool, desc, d, p, x0, y0, z0, tid);
    const int er = hs.er, ec = hs.ec;
    const T* ep = hs.p;
    const int64_t es = hs.stride;
    T* const myc = rc + tid;                     // ring slot s: myc[s * kN]
    T* const mye = re + (tid < kEr ? tid : 0);   // ring slot s: mye[s * kEr]
    int next = z0;                               // the next iteration to copy
    auto issue = [&](int s) {
        if (next < z1) {
            if (kind == 1) cp_async<sizeof(T)>(myc + s * kN, next + 1 == z1 ? zhi : sp);
            else if (kind == 2) cp_async<sizeof(T)>(myc + s * kN, sp);
            if (er >= 0) cp_async<sizeof(T)>(mye + s * kEr, ep);
        }
        cp_async_commit();  // one group per iteration, empty past the range
        sp += ss;
        ep += es;
        ++next;
    };
#pragma unroll
    for (int i = 0; i < RD - 1; ++i) issue(i);

    int s = 0;  // ring slot of iteration k; iteration k + RD - 1 goes to s - 1
#pragma unroll 2
    for (int k = z0; k < z1; ++k) {
        issue(s == 0 ? RD - 1 : s - 1);
        cp_async_wait<RD - 1>();  // this thread's copies for iteration k have landed
        E* buf = sm + (k & 1) * ((kTY + 2) * kSW);
        E* slot = buf + (ty + 1) * kSW + tx + 1;
        if (kind == 1) *slot = wc;
        else if (kind == 2) *slot = myc[s * kN];
        if (er >= 0) buf[er * kSW + ec] = mye[s * kEr];
        __syncthreads();
        if (kind == 1) {
            const E wzp = myc[s * kN];
            const int sc = (ty + 1) * kSW + tx + 1;
            pool[oidx + k * plane] = mean7<T, 0>(wc, buf[sc - 1], buf[sc + 1], buf[sc - kSW], buf[sc + kSW], wzm, wzp);
            wzm = wc;
            wc = wzp;
        }
        s = s == RD - 1 ? 0 : s + 1;
    }
    cp_async_wait<0>();  // only empty groups remain; the ring is free for the next tile
}

// The two-plane engine: the engine above, two planes per step. Each thread
// computes cells (k, k+1) of its column between one pair of barriers, so the
// per-plane bookkeeping (copies, waits, barrier, addressing) is shared by two
// cells and the two cells' integer chains interleave. The exchange buffer
// holds two planes, double-buffered, of frame values (each value converted
// once); the rings work as in the single-plane engine (RD even), with the
// halo ring spread over two threads per slot (one plane each) where the CTA
// has the threads. A range with an odd number of planes ends with a
// single-plane step; cells the frame cannot hold go to the slow list.
// Ops it runs: the exact mean and the residuals (the sequential rule keeps
// the single-plane engine: it is bound by the binary64 pipe either way).
template <int OP>
constexpr bool kPairOp = OP == OP_EXACT || OP == OP_RES || OP == OP_RES32;

template <int OP>
using PairElem = std::conditional_t<OP == OP_RES32, int64_t, frame::W96>;

template <typename T, int OP, int TW>
__host__ __device__ constexpr int pair_smem_bytes()
{
    return 4 * ((kNT<T> / TW + 2) * (TW + 2) + 1) * (int)sizeof(PairElem<OP>);
}

template <typename T, int OP, int TW, int RD>
__host__ __device__ constexpr int pair_engine_bytes()
{
    return pair_smem_bytes<T, OP, TW>() + RD * (kNT<T> + ring_extra<T, TW>()) * (int)sizeof(T);
}

// cp.async of one 8- or 4-byte value, issued only when `on` (a predicated
// instruction, no branch).
template <int N>
__device__ __forceinline__ void cp_async_if(uint32_t dst, const void* src, bool on)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q cp.async.ca.shared.global [%0], [%1], %3;\n\t}\n" ::"r"(dst),
        "l"(src), "r"((int)on), "n"(N)
        : "memory");
}

// As cp_async_if, with a compile-time byte offset added to the shared address.
template <int N, int OFF>
__device__ __forceinline__ void cp_async_if_off(uint32_t dst, const void* src, bool on)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q cp.async.ca.shared.global [%0+%4], [%1], %3;\n\t}\n" ::"r"(dst),
        "l"(src), "r"((int)on), "n"(N), "n"(OFF)
        : "memory");
}

// cp.async of N bytes to a shared address plus a compile-time offset,
// unconditionally.
template <int N, int OFF>
__device__ __forceinline__ void cp_async_off(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0+%2], [%1], %3;\n" ::"r"(dst), "l"(src), "n"(OFF), "n"(N) : "memory");
}

template <typename T, int OP, bool PULL, bool CG, int RD, int TW>
__device__ double tile_engine_pair(T* __restrict__ pool, const BlockDesc* __restrict__ desc,
                                   const int32_t* __restrict__ frame_e, int b, int p, int x0, int y0, int z0, int z1,
                                   unsigned char* smraw, SlowList* slow)
{
    static_assert(kPairOp<OP>, "op");
    using E = PairElem<OP>;
    constexpr int kN = kNT<T>, kTX = TW, kTY = kN / TW, kSW = TW + 2, kEr = ring_extra<T, TW>();
    constexpr int kPlane = (kTY + 2) * kSW + 1;  // + one slot written by threads without a halo slot
    constexpr uint32_t kRowC = kN * sizeof(T), kRowE = kEr * sizeof(T);
    static_assert(RD >= 4 && RD % 2 == 0, "ring depth");
    E* const sm = (E*)smraw;                                   // [2 buffers][2 planes][kPlane]
    T* const rc = (T*)(smraw + pair_smem_bytes<T, OP, TW>());  // [RD][kN]
    T* const re = rc + RD * kN;                                // [RD][kEr]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    // OP_RES32: eref is the binary32 exponent field + 1 (frame_e holds the
    // binary64 field of the largest value)
    const int eref = OP == OP_RES32 ? frame_e[d.inst] + 1 - 896 : frame_e[d.inst] + 1;
    bool bad = false;                    // OP_RES32: a value outside the 64-bit frame
    uint64_t q0 = 0u, q1 = 0u, q2 = 0u;  // OP_RES32: this thread's sum of L^2 in frame units
    double acc = 0.0;                    // OP_RES: this thread's sum of L^2
    // a value as an exchange element (its frame value)
    auto cvt = [&](T v, int er) -> E {
        if constexpr (OP == OP_RES32) {
            bool ok;
            const int64_t w = frame::of32((float)v, er, ok);
            bad |= !ok;
            return w;
        } else {
            return frame::of((double)v, er);
        }
    };
    const bool top_ok = eref >= 7;                          // frame::mean7_top applies
    const uint32_t scale_hi = (uint32_t)(eref - 1081) << 20;  // its scale 2^(25 + eref - 1106)
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const int x = x0 + tx, y = y0 + ty;
    const int64_t plane = d.plane;
    if (tid == 0) slow->n = 0;

    // own stream: the plane above the current one, planes z0+1 .. z1-1 copied
    // (kind 1: an interior column, whose plane z1 is held in a register; kind
    // 2: a halo cell inside the tile); the current plane is carried
    const bool k1 = x < bx && y < by;
    const bool k2 = (x == bx && y < by) || (y == by && x < bx);
    const T* osrc = pool;
    int64_t ostr = 0;
    int olim = z0;  // copies for plane-iterations below olim
    T zhiv = T(0);
    T* out = pool;
    E wzm{}, wc{};
    if (k1) {
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        osrc = col + (z0 + 1) * plane;
        ostr = plane;
        olim = z1 - 1;
        zhiv = ldv<T, CG>(z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : col + z1 * plane);
        out = pool + cell_index<T>(d, p ^ 1, x, y, z0);
        const T* zlo = z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : col + (z0 - 1) * plane;
        wzm = cvt(ldv<T, CG>(zlo), eref);
        wc = cvt(ldv<T, CG>(col + z0 * plane), eref);
    } else if (k2) {
        // a halo cell inside the tile streams like an interior column (its
        // own plane carried, the plane above copied), without computing
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, x, y);
        osrc = s.p + (z0 + 1) * s.stride;
        ostr = s.stride;
        olim = z1 - 1;
        wc = cvt(ldv<T, CG>(s.p + z0 * s.stride), eref);
    }
    // halo-ring slots: with kSplit (2 kEr threads available) thread
    // (hq, hj) = (tid / kEr, tid % kEr) streams slot hj for the planes of
    // parity hq, one copy and one conversion per step; otherwise thread hj =
    // tid < kEr streams slot hj for both planes of a step
    constexpr bool kSplit = 2 * kEr <= kN;
    constexpr int kHT = kSplit ? 2 * kEr : kEr;  // threads with a halo role
    const int hq = kSplit && tid >= kEr ? 1 : 0;
    const int hj = tid - hq * kEr;
    const HaloSlot<T> hs = halo_slot<T, PULL, TW>(pool, desc, d, p, x0, y0, z0, tid < kHT ? hj : kN);
    const bool hv = hs.er >= 0;
    const int hslot = (hv ? hs.er * kSW + hs.ec : kPlane - 1) + hq * kPlane;  // in buffer hq of the pair
    const int64_t hstr = hs.stride;
    const T* hsrc = hs.p + hq * hstr;
    const int hlim = hv ? z1 : z0;
    // a warp with a halo role (from a vote, so the compiler treats the
    // branches on it as warp-uniform)
    const bool halo_warp = __any_sync(0xffffffffu, tid < kHT);
    const int own = (ty + 1) * kSW + tx + 1;
    const uint32_t rc_s = (uint32_t)__cvta_generic_to_shared(rc + tid);
    const T* const mye = re + (tid < kHT ? hj : 0) + hq * kEr;  // ring slot s: mye[s * kEr]
    const uint32_t re_s = (uint32_t)__cvta_generic_to_shared(mye);
    int next = z0;  // the next plane-iteration to copy
    auto copy_pair = [&](int sl) {  // plane-iterations next, next + 1 into slots sl, sl + 1
        cp_async_if<sizeof(T)>(rc_s + sl * kRowC, osrc, next < olim);
        cp_async_if<sizeof(T)>(rc_s + (sl + 1) * kRowC, osrc + ostr, next + 1 < olim);
        if (halo_warp) {  // warps without a halo role issue no halo copies
            if constexpr (kSplit) {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, next + hq < hlim);
            } else {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, next < hlim);
                cp_async_if<sizeof(T)>(re_s + (sl + 1) * kRowE, hsrc + hstr, next + 1 < hlim);
            }
            hsrc += 2 * hstr;
        }
        cp_async_commit();
        osrc += 2 * ostr;
        next += 2;
    };
#pragma unroll
    for (int i = 0; i < RD - 2; i += 2) copy_pair(i);
    __syncthreads();  // slow->n = 0 visible before any append

    int s = 0;  // ring slot of plane-iteration k (even)
    int bsel = 0;
    auto step = [&](auto two_c, auto last_c, int k) {
        constexpr bool TWO = decltype(two_c)::value;
        constexpr bool LAST = decltype(last_c)::value;  // plane z1 may be among k+1, k+2
        copy_pair(s == 0 ? RD - 2 : s - 2);
        cp_async_wait<RD / 2 - 1>();  // this thread's copies for k, k+1 have landed
        E* const b0 = sm + bsel * (2 * kPlane);
        E* const b1 = b0 + kPlane;
        const T v0 = rc[s * kN + tid];
        const T v1 = rc[(s + 1) * kN + tid];
        // planes k+1, k+2 of the own column (plane z1 from the register)
        const E c0 = cvt((LAST && k + 1 >= z1 ? zhiv : v0), eref);
        const E c1 = cvt((LAST && k + 2 >= z1 ? zhiv : v1), eref);
        b0[own] = wc;
        if (TWO) b1[own] = c0;
        if (halo_warp) {
            if constexpr (kSplit) {
                if (TWO || hq == 0) b0[hslot] = cvt(mye[s * kEr], eref);
            } else {
                b0[hslot] = cvt(mye[s * kEr], eref);
                if (TWO) b1[hslot] = cvt(mye[(s + 1) * kEr], eref);
            }
        }
        __syncthreads();
        if constexpr (OP == OP_RES32) {
            // L = xm + xp + ym + yp + zm + zp - 6c, exact in the 64-bit frame
            const int64_t L0 = b0[own - 1] + b0[own + 1] + b0[own - kSW] + b0[own + kSW] + wzm + c0 - 6 * wc;
            if (k1) frame::add_square(L0, q0, q1, q2);
            if (TWO) {
                const int64_t L1 = b1[own - 1] + b1[own + 1] + b1[own - kSW] + b1[own + kSW] + wc + c1 - 6 * c0;
                if (k1) frame::add_square(L1, q0, q1, q2);
            }
        } else if constexpr (OP == OP_RES) {
            double o;
            const bool ok0 = frame::laplacian(wc, b0[own - 1], b0[own + 1], b0[own - kSW], b0[own + kSW], wzm, c0, eref, o);
            if (k1 && ok0) acc = fma(o, o, acc);
            if (k1 && !ok0) {
                const int i = atomicAdd(&slow->n, 1);
                if (i < kSlowMax) slow->cell[i] = ((uint32_t)k << 9) | (uint32_t)tid;
            }
            if (TWO) {
                const bool ok1 = frame::laplacian(c0, b1[own - 1], b1[own + 1], b1[own - kSW], b1[own + kSW], wc, c1, eref, o);
                if (k1 && ok1) acc = fma(o, o, acc);
                if (k1 && !ok1) {
                    const int i = atomicAdd(&slow->n, 1);
                    if (i < kSlowMax) slow->cell[i] = ((uint32_t)(k + 1) << 9) | (uint32_t)tid;
                }
            }
        } else {
            uint32_t a0, a1, a2, e0 = 0u, e1 = 0u, e2 = 0u;
            if (TWO) {  // planes k and k+1 share the term wc + c0
                const E t = frame::add(wc, c0);
                frame::sum6(t, b0[own - 1], b0[own + 1], b0[own - kSW], b0[own + kSW], wzm, a0, a1, a2);
                frame::sum6(t, b1[own - 1], b1[own + 1], b1[own - kSW], b1[own + kSW], c1, e0, e1, e2);
            } else {
                frame::sum7(wc, b0[own - 1], b0[own + 1], b0[own - kSW], b0[own + kSW], wzm, c0, a0, a1, a2);
            }
            // the fixed-shift mean when every computing lane's sums lie in the
            // top binades of the frame (nearly always), else the general one;
            // each branch stores its own results
            const bool top = top_ok && frame::sum_in_top(a2) && (!TWO || frame::sum_in_top(e2));
            if (__all_sync(0xffffffffu, top || !k1)) {
                const double o0 = frame::mean7_top(a0, a1, a2, scale_hi);
                if (k1) out[0] = (T)o0;
                if (TWO) {
                    const double o1 = frame::mean7_top(e0, e1, e2, scale_hi);
                    if (k1) out[plane] = (T)o1;
                }
            } else {
                double o0, o1;
                const bool ok0 = frame::mean7_of_sum(a0, a1, a2, eref, o0);
                if (k1 && ok0) out[0] = (T)o0;
                if (k1 && !ok0) {
                    const int i = atomicAdd(&slow->n, 1);
                    if (i < kSlowMax) slow->cell[i] = ((uint32_t)k << 9) | (uint32_t)tid;
                }
                if (TWO) {
                    const bool ok1 = frame::mean7_of_sum(e0, e1, e2, eref, o1);
                    if (k1 && ok1) out[plane] = (T)o1;
                    if (k1 && !ok1) {
                        const int i = atomicAdd(&slow->n, 1);
                        if (i < kSlowMax) slow->cell[i] = ((uint32_t)(k + 1) << 9) | (uint32_t)tid;
                    }
                }
            }
        }
        out += 2 * plane;
        wzm = c0;
        wc = c1;
        s = s == RD - 2 ? 0 : s + 2;
        bsel ^= 1;
    };
    int k = z0;
    // two steps per pass (the carried planes alternate registers), planes
    // k+1 .. k+4 below z1 (all from the ring); the last one to four planes
    // after the loop
    for (; k + 4 < z1; k += 4) {
        step(std::true_type{}, std::false_type{}, k);
        step(std::true_type{}, std::false_type{}, k + 2);
    }
    if (k + 2 < z1) {
        step(std::true_type{}, std::false_type{}, k);
        k += 2;
    }
    if (k + 1 < z1) step(std::true_type{}, std::true_type{}, k);
    else if (k < z1) step(std::false_type{}, std::true_type{}, k);
    cp_async_wait<0>();
    if constexpr (OP == OP_RES32) {
        // L^2 was summed exactly in units of 2^(2 (eref - 186)); a value
        // outside the frame anywhere in the tile redoes the whole tile with
        // the exact per-cell routines
        acc = frame::u192_to_double_scaled(q0, q1, q2, 2 * (eref - 186));
        if (__syncthreads_or(bad)) {
            if (tid == 0) slow->n = kSlowMax + 1;
        }
        return slow_cells<T, OP_RES, PULL, CG, TW>(pool, desc, d, b, p, x0, y0, z0, z1, k1, x, y, 0, acc, slow);
    } else if constexpr (OP == OP_RES) {
        return slow_cells<T, OP_RES, PULL, CG, TW>(pool, desc, d, b, p, x0, y0, z0, z1, k1, x, y, 0, acc, slow);
    } else {
        return slow_cells<T, OP_EXACT, PULL, CG, TW>(pool, desc, d, b, p, x0, y0, z0, z1, k1, x, y,
                                                     cell_index<T>(d, p ^ 1, x, y, 0), 0.0, slow);
    }
}

// ------------------------------------------------------- 64-bit frame engine
// The correctly rounded mean with the grid's values held as 64-bit frame
// integers (nframe): 8 bytes per exchange-plane value, one 64-bit sum per
// cell, one normalising division by 7. A step whose tile plane holds a value
// outside the frame's nine binades (a tile-wide vote at the step's barrier)
// is redone in the 96-bit frame from the raw values, which are still in the
// prefetch rings (own planes k+1, k+2 and the halo ring) or in global memory
// (own planes k-1, k); the next step tries the 64-bit frame again.

// One halo-ring slot per thread for tid < 2 (TW + TY), as halo_slot, except
// that a tile overhanging the block edge takes its right column and bottom
// row of halo at the edge itself (x = bx, y = by), so every own-column lane
// of the engine is an interior cell.
template <bool PULL, int TW>
__device__ __forceinline__ HaloSlot<double> halo_slot_edge(const double* pool, const BlockDesc* desc,
                                                           const BlockDesc& d, int p, int x0, int y0, int z0, int tid)
{
    using T = double;
    constexpr int kTW = TW, kTY = kNT<T> / TW;
    const int bx = d.ext[0], by = d.ext[1];
    HaloSlot<T> h{-1, 0, pool, 0};
    if (tid >= ring_extra<T, TW>()) return h;
    const int xr = min(x0 + kTW, bx), yb = min(y0 + kTY, by);  // the right column and bottom row
    int hx, hy;
    if (tid < kTW) {
        hx = x0 + tid;
        hy = y0 - 1;
        h.er = hx < bx ? 0 : -1;
        h.ec = tid + 1;
    } else if (tid < 2 * kTW) {
        const int c = tid - kTW;
        hx = x0 + c;
        hy = yb;
        h.er = hx < bx ? yb - y0 + 1 : -1;
        h.ec = c + 1;
    } else if (tid < 2 * kTW + kTY) {
        const int r = tid - 2 * kTW;
        hx = x0 - 1;
        hy = y0 + r;
        h.er = hy < by ? r + 1 : -1;
        h.ec = 0;
    } else {
        const int r = tid - 2 * kTW - kTY;
        hx = xr;
        hy = y0 + r;
        h.er = hy < by ? r + 1 : -1;
        h.ec = xr - x0 + 1;
    }
    if (h.er >= 0) {
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, hx, hy);
        h.p = s.p + z0 * s.stride;
        h.stride = s.stride;
    }
    return h;
}

template <int TW>
__host__ __device__ constexpr int narrow_plane()
{
    return (kNT<double> / TW + 2) * (TW + 2) + 1;  // + one slot written by lanes without a slot of their own
}

// [2 buffers][2 planes][plane] 64-bit values, then one 96-bit plane (the
// fallback step's second plane; its first is the current 64-bit buffer).
template <int TW>
__host__ __device__ constexpr int narrow_smem_bytes()
{
    return 4 * narrow_plane<TW>() * 8 + narrow_plane<TW>() * (int)sizeof(frame::W96);
}

template <int TW, int RD>
__host__ __device__ constexpr int narrow_engine_bytes()
{
    return narrow_smem_bytes<TW>() + RD * (kNT<double> + ring_extra<double, TW>()) * (int)sizeof(double);
}

// The exact mean over one tile of block b (TW x 256/TW columns, planes z0 ..
// z1-1), reading buffer p and writing buffer p^1. PULL: halo values come
// from the neighbouring blocks (the fused and persistent forms); otherwise
// from the block's ghost layer (only for blocks whose ghost layer the
// unfused flow has filled). Each thread owns one column and computes two
// planes per step; copies run RD - 2 planes ahead.
template <bool PULL, bool CG, int RD, int TW>
__device__ void tile_engine_narrow(double* __restrict__ pool, const BlockDesc* __restrict__ desc,
                                   const int32_t* __restrict__ frame_e, int b, int p, int x0, int y0, int z0, int z1,
                                   unsigned char* smraw, SlowList* slow)
{
    using T = double;
    using W = frame::W96;
    constexpr int kN = kNT<T>, kTX = TW, kTY = kN / TW, kSW = TW + 2, kEr = ring_extra<T, TW>();
    constexpr int kPlane = narrow_plane<TW>();
    constexpr uint32_t kRowC = kN * sizeof(T), kRowE = kEr * sizeof(T);
    static_assert(RD >= 4 && RD % 2 == 0, "ring depth");
    static_assert(2 * kPlane * 8 == kPlane * (int)sizeof(W), "a 64-bit plane pair holds one 96-bit plane");
    uint64_t* const nsm = (uint64_t*)smraw;                   // [2 buffers][2 planes][kPlane]
    W* const wx = (W*)(smraw + 4 * kPlane * 8);               // [kPlane]
    T* const rc = (T*)(smraw + narrow_smem_bytes<TW>());      // [RD][kN]
    T* const re = rc + RD * kN;                               // [RD][kEr]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int eref = frame_e[d.inst] + 1;
    // the 64-bit frame needs eref >= 13 (normal results); below that every
    // step takes the 96-bit frame
    const bool nok = eref >= 13;
    const uint32_t elo = nframe::elo_hi(eref), nscale = nframe::scale_hi(eref);
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const int x = x0 + tx, y = y0 + ty;
    const int64_t plane = d.plane;
    if (tid == 0) slow->n = 0;

    // own stream (interior columns only): the plane above the current one,
    // planes z0+1 .. z1-1 copied; plane z1 is held in a register; the two
    // current planes are carried as frame integers with their window flags
    const bool k1 = x < bx && y < by;
    const T* osrc = pool;
    int olim = z0;
    T zhiv = T(0);
    T* out = pool;
    uint64_t wzm = 0u, wc = 0u;
    bool gzm = true, gc = true;
    if (k1) {
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        osrc = col + (z0 + 1) * plane;
        olim = z1 - 1;
        zhiv = ldv<T, CG>(z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : col + z1 * plane);
        out = pool + cell_index<T>(d, p ^ 1, x, y, z0);
        const T* zlo = z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : col + (z0 - 1) * plane;
        wzm = nframe::of0(ldv<T, CG>(zlo), elo, gzm);
        wc = nframe::of(ldv<T, CG>(col + z0 * plane), elo, gc);
    }
    bool gzh;
    const uint64_t zhn = nframe::of0(zhiv, elo, gzh);
    // halo-ring slots, as in the 96-bit engine (kSplit: two threads per
    // slot, one plane parity each)
    constexpr bool kSplit = 2 * kEr <= kN;
    constexpr int kHT = kSplit ? 2 * kEr : kEr;
    const int hq = kSplit && tid >= kEr ? 1 : 0;
    const int hj = tid - hq * kEr;
    const HaloSlot<T> hs = halo_slot_edge<PULL, TW>(pool, desc, d, p, x0, y0, z0, tid < kHT ? hj : kN);
    const bool hv = hs.er >= 0;
    const int hbase = hv ? hs.er * kSW + hs.ec : kPlane - 1;  // slot within a plane
    const int hslot = hbase + hq * kPlane;                    // within a buffer's plane pair
    const int64_t hstr = hs.stride;
    const T* hsrc = hs.p + hq * hstr;
    const int hlim = hv ? z1 : z0;
    const bool halo_warp = __any_sync(0xffffffffu, tid < kHT);
    const int own = (ty + 1) * kSW + tx + 1;
    const int ownw = k1 ? own : kPlane - 1;  // lanes outside the block store into the spare slot
    const uint32_t rc_s = (uint32_t)__cvta_generic_to_shared(rc + tid);
    const T* const mye = re + (tid < kHT ? hj : 0) + hq * kEr;
    const uint32_t re_s = (uint32_t)__cvta_generic_to_shared(mye);
    int next = z0;
    auto copy_pair = [&](int sl) {
        cp_async_if<sizeof(T)>(rc_s + sl * kRowC, osrc, next < olim);
        cp_async_if<sizeof(T)>(rc_s + (sl + 1) * kRowC, osrc + plane, next + 1 < olim);
        if (halo_warp) {
            if constexpr (kSplit) {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, next + hq < hlim);
            } else {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, next < hlim);
                cp_async_if<sizeof(T)>(re_s + (sl + 1) * kRowE, hsrc + hstr, next + 1 < hlim);
            }
            hsrc += 2 * hstr;
        }
        cp_async_commit();
        osrc += 2 * plane;
        next += 2;
    };
#pragma unroll
    for (int i = 0; i < RD - 2; i += 2) copy_pair(i);
    __syncthreads();  // slow->n = 0 visible before any append

    int s = 0;  // ring slot of plane-iteration k (even)
    int bsel = 0;
    auto step = [&](auto two_c, auto last_c, int k) {
        constexpr bool TWO = decltype(two_c)::value;
        constexpr bool LAST = decltype(last_c)::value;  // plane z1 may be among k+1, k+2
        copy_pair(s == 0 ? RD - 2 : s - 2);
        cp_async_wait<RD / 2 - 1>();
        uint64_t* const n0 = nsm + bsel * (2 * kPlane);
        uint64_t* const n1 = n0 + kPlane;
        bool g0, g1 = true;
        uint64_t c0 = nframe::of(rc[s * kN + tid], elo, g0);
        if (LAST && k + 1 >= z1) {
            c0 = zhn;
            g0 = gzh;
        }
        uint64_t c1 = 0u;
        if (TWO) {
            c1 = nframe::of(rc[(s + 1) * kN + tid], elo, g1);
            if (LAST && k + 2 >= z1) {
                c1 = zhn;
                g1 = gzh;
            }
        }
        n0[ownw] = wc;
        if (TWO) n1[ownw] = c0;
        bool gh = true;
        if (halo_warp) {
            if constexpr (kSplit) {
                if (TWO || hq == 0) n0[hslot] = nframe::of0(mye[s * kEr], elo, gh);
            } else {
                bool gh1;
                n0[hslot] = nframe::of0(mye[s * kEr], elo, gh);
                if (TWO) {
                    n1[hslot] = nframe::of0(mye[(s + 1) * kEr], elo, gh1);
                    gh = gh && gh1;
                }
            }
        }
        const bool bad = !nok || (k1 && !(gzm && gc && g0 && g1)) || (hv && !gh);
        if (!__syncthreads_or(bad)) {
            // every value of the step is in the 64-bit frame
            const uint64_t t = wc + c0;
            const uint64_t S0 = t + n0[own - 1] + n0[own + 1] + n0[own - kSW] + n0[own + kSW] + wzm;
            if (k1) out[0] = nframe::mean7(S0, nscale);
            if (TWO) {
                const uint64_t S1 = t + n1[own - 1] + n1[own + 1] + n1[own - kSW] + n1[own + kSW] + c1;
                if (k1) out[plane] = nframe::mean7(S1, nscale);
            }
        } else {
            // the step in the 96-bit frame: plane k in the current 64-bit
            // buffer pair (no thread reads it any more: the decision came at
            // the barrier all of them passed), plane k+1 in the spare plane
            W* const A = (W*)n0;
            W* const B = wx;
            W fzm{}, fc{}, f0{}, f1{};
            if (k1) {
                // own planes k and k-1 from global memory, k+1 and k+2 from
                // the ring (or the plane-z1 register)
                const T* pk = osrc - (int64_t)(RD + 1) * plane;
                const T* pzm = (k == z0 && z0 == 0) ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : pk - plane;
                fc = frame::of(ldv<T, CG>(pk), eref);
                fzm = frame::of(ldv<T, CG>(pzm), eref);
                f0 = frame::of((LAST && k + 1 >= z1) ? zhiv : rc[s * kN + tid], eref);
                if (TWO) f1 = frame::of((LAST && k + 2 >= z1) ? zhiv : rc[(s + 1) * kN + tid], eref);
            }
            A[ownw] = fc;
            if (TWO) B[ownw] = f0;
            if (halo_warp) {
                if constexpr (kSplit) {
                    if (TWO || hq == 0) (hq ? B : A)[hbase] = frame::of(mye[s * kEr], eref);
                } else {
                    A[hbase] = frame::of(mye[s * kEr], eref);
                    if (TWO) B[hbase] = frame::of(mye[(s + 1) * kEr], eref);
                }
            }
            __syncthreads();
            uint32_t a0, a1, a2;
            double o;
            frame::sum7(fc, A[own - 1], A[own + 1], A[own - kSW], A[own + kSW], fzm, f0, a0, a1, a2);
            const bool ok0 = frame::mean7_of_sum(a0, a1, a2, eref, o);
            if (k1 && ok0) out[0] = o;
            if (k1 && !ok0) {
                const int i = atomicAdd(&slow->n, 1);
                if (i < kSlowMax) slow->cell[i] = ((uint32_t)k << 9) | (uint32_t)tid;
            }
            if (TWO) {
                frame::sum7(f0, B[own - 1], B[own + 1], B[own - kSW], B[own + kSW], fc, f1, a0, a1, a2);
                const bool ok1 = frame::mean7_of_sum(a0, a1, a2, eref, o);
                if (k1 && ok1) out[plane] = o;
                if (k1 && !ok1) {
                    const int i = atomicAdd(&slow->n, 1);
                    if (i < kSlowMax) slow->cell[i] = ((uint32_t)(k + 1) << 9) | (uint32_t)tid;
                }
            }
        }
        out += 2 * plane;
        wzm = c0;
        gzm = g0;
        wc = c1;
        gc = g1;
        s = s == RD - 2 ? 0 : s + 2;
        bsel ^= 1;
    };
    int k = z0;
    for (; k + 4 < z1; k += 4) {
        step(std::true_type{}, std::false_type{}, k);
        step(std::true_type{}, std::false_type{}, k + 2);
    }
    if (k + 2 < z1) {
        step(std::true_type{}, std::false_type{}, k);
        k += 2;
    }
    if (k + 1 < z1) step(std::true_type{}, std::true_type{}, k);
    else if (k < z1) step(std::false_type{}, std::true_type{}, k);
    cp_async_wait<0>();
    slow_cells<T, OP_EXACT, PULL, CG, TW>(pool, desc, d, b, p, x0, y0, z0, z1, k1, x, y,
                                          cell_index<T>(d, p ^ 1, x, y, 0), 0.0, slow);
}

// ----------------------------------------- two-column 64-bit frame engine
// The 64-bit frame engine with each thread owning an x-adjacent pair of
// columns (blocks of even x extent): a tile of TW x 512/TW cells per plane
// for 256 threads. The pair moves as one 16-byte value everywhere (copy into
// the ring, ring load, exchange-plane store, result store) and its two cells
// share partial sums, so the per-step work of copies, addressing and the
// loop is spread over four cells. The ring holds four planes, so with two
// steps per pass every ring slot and exchange buffer is a compile-time offset.
// Exchange-plane row: a spare slot, the left halo, the TW cells (pairs on
// 16-byte boundaries), the right halo, a spare slot.
constexpr int kRing2 = 4;

template <int TW>
__host__ __device__ constexpr int n2_rows()
{
    return 2 * kNT<double> / TW;
}

template <int TW>
__host__ __device__ constexpr int n2_ring_extra()
{
    return 2 * TW + 2 * n2_rows<TW>();
}

template <int TW>
__host__ __device__ constexpr int n2_plane()
{
    return (n2_rows<TW>() + 2) * (TW + 4) + 2;  // + a spare pair for lanes without a slot
}

template <int TW>
__host__ __device__ constexpr int n2_engine_bytes()
{
    // exchange planes, the own-pair ring plus one slot for plane z1, the halo ring
    return 4 * n2_plane<TW>() * 8 + ((kRing2 + 1) * 2 * kNT<double> + kRing2 * n2_ring_extra<TW>()) * (int)sizeof(double);
}

// The pair (x, x+1) of column (x, y) at plane -1 (zface 4) or bz (zface 5):
// from the neighbouring block, the Dirichlet pair, or (not PULL) the block's
// ghost layer. Always 16-byte aligned (x even, rows on 128-byte boundaries).
template <bool PULL>
__device__ __forceinline__ const double* z_pair_source(const double* pool, const BlockDesc* desc, const BlockDesc& d,
                                                       int p, int x, int y, int zface)
{
    if constexpr (PULL) {
        if (d.nbr[zface] < 0) return d.bc2[zface];
    }
    return z_source<double, PULL>(pool, desc, d, p, x, y, zface);
}

template <bool CG>
__device__ __forceinline__ double2 ld_pair(const double* p)
{
    if constexpr (CG) return __ldcg((const double2*)p);
    else return __ldg((const double2*)p);
}

// One halo-ring slot per thread for tid < 2 (TW + TY) of the two-column
// tile (rows y0-1 and the bottom edge, columns x0-1 and the right edge, the
// edges taken at the block boundary where the tile overhangs it).
template <bool PULL, int TW>
__device__ __forceinline__ HaloSlot<double> halo_slot_pair(const double* pool, const BlockDesc* desc,
                                                           const BlockDesc& d, int p, int x0, int y0, int z0, int tid)
{
    using T = double;
    constexpr int kTW = TW, kTY = n2_rows<TW>(), kSW = TW + 4;
    const int bx = d.ext[0], by = d.ext[1];
    HaloSlot<T> h{-1, 0, pool, 0};
    if (tid >= n2_ring_extra<TW>()) return h;
    const int xr = min(x0 + kTW, bx), yb = min(y0 + kTY, by);
    int hx, hy;
    // (er, ec) here is the slot's row and its index within the row
    if (tid < kTW) {
        hx = x0 + tid;
        hy = y0 - 1;
        h.er = hx < bx ? 0 : -1;
        h.ec = 2 + tid;
    } else if (tid < 2 * kTW) {
        const int c = tid - kTW;
        hx = x0 + c;
        hy = yb;
        h.er = hx < bx ? yb - y0 + 1 : -1;
        h.ec = 2 + c;
    } else if (tid < 2 * kTW + kTY) {
        const int r = tid - 2 * kTW;
        hx = x0 - 1;
        hy = y0 + r;
        h.er = hy < by ? r + 1 : -1;
        h.ec = 1;
    } else {
        const int r = tid - 2 * kTW - kTY;
        hx = xr;
        hy = y0 + r;
        h.er = hy < by ? r + 1 : -1;
        h.ec = 2 + xr - x0;
    }
    static_assert(kSW == kTW + 4, "row layout");
    if (h.er >= 0) {
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, hx, hy);
        h.p = s.p + z0 * s.stride;
        h.stride = s.stride;
    }
    return h;
}

// After the tile's loop: the cells recorded in the slow list (or, when it
// overflowed, every cell of the tile) with the exact per-cell routine.
// Slow-list entries of the two-column engine: (k << 10) | (tid << 1) | cell.
// The exponent field of |v|.
__device__ __forceinline__ int exp_field(double v) { return (int)((dbits(v) >> 52) & 0x7FFull); }

template <bool PULL, bool CG, int TW>
__device__ __forceinline__ void n2_slow_cells(double* pool, const BlockDesc* desc, const BlockDesc& d, int b, int p,
                                              int x0, int y0, int z0, int z1, bool k1, int x, int y, SlowList* slow,
                                              int eref, int& lzm)
{
    constexpr int kTP = TW / 2;
    __syncthreads();
    const int n = slow->n;
    if (n == 0) return;
    const int tid = threadIdx.x;
    if (n <= kSlowMax) {
        for (int i = tid; i < n; i += kNT<double>) {
            const uint32_t c = slow->cell[i];
            const int kk = (int)(c >> 10), t = (int)((c >> 1) & 511u), cell = (int)(c & 1u);
            const int cx = x0 + 2 * (t % kTP) + cell, cy = y0 + t / kTP;
            const double v = exact_cell<double, PULL, CG, false>(pool, desc, b, p, cx, cy, kk);
            pool[cell_index<double>(d, p ^ 1, cx, cy, kk)] = v;
            lzm = min(lzm, eref - exp_field(v));
        }
    } else if (k1) {
        for (int kk = z0; kk < z1; ++kk)
            for (int cell = 0; cell < 2; ++cell) {
                const double v = exact_cell<double, PULL, CG, false>(pool, desc, b, p, x + cell, y, kk);
                pool[cell_index<double>(d, p ^ 1, x + cell, y, kk)] = v;
                lzm = min(lzm, eref - exp_field(v));
            }
    }
}

// The exact mean over one two-column tile of block b (bx even): columns x0 ..
// x0+TW-1, rows y0 .. y0+512/TW-1, planes z0 .. z1-1; buffer p read, p^1
// written.
// Steps come in two kinds. The hot step (two planes below z1, compile-time
// ring phase) has no path but the 64-bit frame: when the tile-wide vote
// finds a value outside it, the step stops before computing and the generic
// step resumes it. The generic step (run-time phase, the last planes of the
// tile, the step after a fallback) falls back to the 96-bit frame itself. The
// 96-bit path thus stays out of the hot loop, whose registers it would
// otherwise take.
// Unit exponent bounds (uin, uout; null: the grid's frame only): uin holds,
// per work unit, an upper bound on the exponent field of the values that
// unit wrote into the buffer read now (all ones where unknown); the tile's
// frame is taken from the largest bound over the units of its block and of
// its six neighbours (the only blocks whose values it reads) and the
// block's Dirichlet values, and never above the grid's frame. At its end the
// tile stores the bound of its own outputs in *uout. The frame only scales
// the integers, so the results do not depend on it.
// What the residual modes return per thread: the exact sum of L^2 of its
// cells in units of 2^(2 (eref - 1084)) (192 bits: each term below 2^128, at
// most 512 of them per thread), and whether a step of
// the tile took the 96-bit frame (the unit's residual is then taken again by
// the two-plane engine).
struct R64Out {
    uint64_t q0, q1, q2;
    bool bad;
};

// RM (residual mode): 0 the update only; 1 the update and, from the same
// 64-bit sums, L = S - 7c of the grid it reads; 2 the residual terms only
// (nothing is written). The residual modes are called with the grid's frame
// (uin null), so whether a unit falls back does not depend on the bounds.
// The frame sources of a unit: its list in fs, or n = -1 where it has none.
struct FrameSources {
    const int32_t* list;
    int n;
};

__device__ __forceinline__ FrameSources frame_sources(const int32_t* fs, const TileUnit& u)
{
    if (!fs || u.fsn < 0) return {nullptr, -1};
    return {fs + u.fs0, u.fsn};
}

template <bool PULL, bool CG, int TW, int RM = 0>
__device__ void tile_engine_narrow2(double* __restrict__ pool, const BlockDesc* __restrict__ desc,
                                    const int32_t* __restrict__ frame_e, int b, int p, int x0, int y0, int z0, int z1,
                                    unsigned char* smraw, SlowList* slow, const uint32_t* uin, uint32_t* uout,
                                    R64Out* ro = nullptr, FrameSources fsrc = {nullptr, -1})
{
    using T = double;
    using W = frame::W96;
    constexpr int RD = kRing2;
    constexpr int kN = kNT<T>, kTP = TW / 2, kSW = TW + 4, kEr = n2_ring_extra<TW>();
    constexpr int kPlane = n2_plane<TW>();
    constexpr uint32_t kRowC = 2 * kN * sizeof(T), kRowE = kEr * sizeof(T);
    static_assert(kEr <= kN, "every halo-ring slot needs a thread");
    static_assert(kPlane % 2 == 0 && kSW % 2 == 0, "pairs on 16-byte boundaries");
    static_assert(4 * kPlane * 8 == 2 * kPlane * (int)sizeof(W), "the four 64-bit planes hold two 96-bit planes");
    uint64_t* const nsm = (uint64_t*)smraw;                 // [2 buffers][2 planes][kPlane]
    T* const rc = (T*)(smraw + 4 * kPlane * 8);             // [RD + 1][kN][2]: the ring, then plane z1
    T* const re = rc + (RD + 1) * 2 * kN;                   // [RD][kEr]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tid = threadIdx.x, tp = tid % kTP, ty = tid / kTP;
    __shared__ uint32_t s_red[kN / 32];
    const int x = x0 + 2 * tp, y = y0 + ty;
    const int plane = (int)d.plane;  // block dims are at most 256: a plane holds fewer than 2^17 elements
    if (tid == 0) {
        slow->n = 0;
        // this unit's bound of the buffer written now: its readers (the
        // previous iteration's tiles of this block and its neighbours) have
        // all finished; the warps fold their bounds into it at the end
        if (uout) *uout = 0u;
    }

    // own pair stream: planes z0+1 .. z1-1 through the ring, plane z1 into its
    // own slot at the start; the two current planes carried as frame integers
    const bool k1 = x < bx && y < by;  // both cells: bx is even
    // lanes without a column keep a fixed, readable source (the pool's first
    // pair), so the hot steps can copy unconditionally
    const T* osrc = pool;
    const int oplane = k1 ? plane : 0;
    int olim = z0;
    T* out = pool;
    uint64_t zmA = 0u, zmB = 0u, cA = 0u, cB = 0u;
    bool gzm = true, gc = true;
    const uint32_t rz_s = (uint32_t)__cvta_generic_to_shared(rc + 2 * (RD * kN + tid));
    double2 zl = make_double2(0.0, 0.0), c00 = make_double2(0.0, 0.0);  // planes z0 - 1, z0 (converted below)
    if (k1) {
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        osrc = col + (int64_t)(z0 + 1) * plane;
        olim = z1 - 1;
        out = pool + cell_index<T>(d, p ^ 1, x, y, z0);
        cp_async_if<16>(rz_s, z1 == bz ? z_pair_source<PULL>(pool, desc, d, p, x, y, 5) : col + (int64_t)z1 * plane,
                        true);
        zl = ld_pair<CG>(z0 == 0 ? z_pair_source<PULL>(pool, desc, d, p, x, y, 4) : col + (int64_t)(z0 - 1) * plane);
        c00 = ld_pair<CG>(col + (int64_t)z0 * plane);
    }
    constexpr bool kSplit = 2 * kEr <= kN;
    constexpr int kHT = kSplit ? 2 * kEr : kEr;
    const int hq = kSplit && tid >= kEr ? 1 : 0;
    const int hj = tid - hq * kEr;
    const HaloSlot<T> hs = halo_slot_pair<PULL, TW>(pool, desc, d, p, x0, y0, z0, tid < kHT ? hj : kN);
    const bool hv = hs.er >= 0;
    const int hbase = hv ? hs.er * kSW + hs.ec : kPlane - 1;
    const int hslot = hbase + hq * kPlane;
    const int hstr = (int)hs.stride;
    const T* hsrc = hs.p + hq * hstr;
    const int hlim = hv ? z1 : z0;
    const bool halo_warp = __any_sync(0xffffffffu, tid < kHT);
    const int own = (ty + 1) * kSW + 2 + 2 * tp;
    const int ownw = k1 ? own : kPlane - 2;
    const uint32_t rc_s = (uint32_t)__cvta_generic_to_shared(rc + 2 * tid);
    const T* const mye = re + (tid < kHT ? hj : 0) + hq * kEr;
    const uint32_t re_s = (uint32_t)__cvta_generic_to_shared(mye);
    const int hvi = hv ? 1 : 0;
    // copies for the plane-iterations j, j + 1 (planes j+1, j+2 of the own
    // pair, planes j, j+1 of the halo ring) into ring slots sl, sl + 1. The
    // hot steps' copies all lie below z1 (j = k + 2 with k + 4 < z1): no
    // bounds to test, only whether the lane has a halo slot.
    auto copy_c = [&](auto sl_c) {  // sl a compile-time constant
        constexpr int sl = decltype(sl_c)::value;
        cp_async_off<16, sl * kRowC>(rc_s, osrc);
        cp_async_off<16, (sl + 1) * kRowC>(rc_s, osrc + oplane);
        if (halo_warp) {
            if constexpr (kSplit) {
                cp_async_if_off<sizeof(T), sl * kRowE>(re_s, hsrc, hvi);
            } else {
                cp_async_if_off<sizeof(T), sl * kRowE>(re_s, hsrc, hvi);
                cp_async_if_off<sizeof(T), (sl + 1) * kRowE>(re_s, hsrc + hstr, hvi);
            }
            hsrc += 2 * hstr;
        }
        cp_async_commit();
        osrc += 2 * oplane;
    };
    auto copy_r = [&](int sl, int j) {  // sl known at run time; j may reach z1
        cp_async_if<16>(rc_s + sl * kRowC, osrc, j < olim);
        cp_async_if<16>(rc_s + (sl + 1) * kRowC, osrc + oplane, j + 1 < olim);
        if (halo_warp) {
            if constexpr (kSplit) {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, j + hq < hlim);
            } else {
                cp_async_if<sizeof(T)>(re_s + sl * kRowE, hsrc, j < hlim);
                cp_async_if<sizeof(T)>(re_s + (sl + 1) * kRowE, hsrc + hstr, j + 1 < hlim);
            }
            hsrc += 2 * hstr;
        }
        cp_async_commit();
        osrc += 2 * oplane;
    };
    copy_r(0, z0);
    // the tile's frame from the exponent bounds (after the first copies and
    // loads are in flight, so their latencies overlap)
    if (uin) {
        uint32_t emax = 0u;
        if (fsrc.n >= 0) {
            // the largest exponent bound of the units this tile reads, and the
            // Dirichlet values of the faces it touches
            for (int i = tid; i < fsrc.n; i += kN) emax = max(emax, __ldcg(uin + fsrc.list[i]));
            if (tid == 0) {
                const bool touch[6] = {x0 == 0, x0 + TW >= bx, y0 == 0, y0 + n2_rows<TW>() >= by, z0 == 0, z1 >= bz};
                for (int j = 0; j < 6; ++j)
                    if (d.nbr[j] < 0 && touch[j]) emax = max(emax, (uint32_t)exp_field(d.bc[j]));
            }
        } else {
            // the largest exponent bound of the blocks this tile reads
            for (int j = 0; j < 7; ++j) {
                const int nb = j == 0 ? b : d.nbr[j - 1];
                if (nb < 0) {
                    if (tid == 0) emax = max(emax, (uint32_t)exp_field(d.bc[j - 1]));
                    continue;
                }
                const BlockDesc& n = desc[nb];
                const int u0 = n.u0, nt = n.ntiles;
                for (int i = tid; i < nt; i += kN) emax = max(emax, __ldcg(uin + u0 + i));
            }
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        if ((tid & 31) == 0) s_red[tid >> 5] = emax;
    }
    __syncthreads();  // slow->n = 0 visible before any append; the warps' exponent bounds
    int eref = frame_e[d.inst] + 1;
    if (uin) {
        uint32_t emax = 0u;
#pragma unroll
        for (int w = 0; w < kN / 32; ++w) emax = max(emax, s_red[w]);
        if (emax < 2047u) eref = min(eref, (int)emax + 1);
    }
    const bool nok = eref >= 13;  // else every step takes the 96-bit frame
    const uint32_t elo = nframe::elo_hi(eref), nscale = nframe::scale_hi(eref);
    int lzm = 64;  // the least leading-zero count of this thread's sums: its results' fields are <= eref - lzm
    if (k1) {
        bool g1, g2;
        zmA = nframe::of0(zl.x, elo, g1);
        zmB = nframe::of0(zl.y, elo, g2);
        gzm = g1 && g2;
        cA = nframe::of(c00.x, elo, g1);
        cB = nframe::of(c00.y, elo, g2);
        gc = g1 && g2;
    }

    // the current step's two new own planes (k+1, k+2) as frame integers
    uint64_t c0A = 0u, c0B = 0u, c1A = 0u, c1B = 0u;
    bool g0 = true, g1 = true;
    // residual modes: this thread's sum of L^2 and whether a step fell back
    [[maybe_unused]] uint64_t rq0 = 0u, rq1 = 0u, rq2 = 0u;
    [[maybe_unused]] bool rbad = false;
    // L = S - 7c, its square added exactly (nframe::add_laplacian_square)
    [[maybe_unused]] auto lsq = [&](uint64_t S, uint64_t c) { nframe::add_laplacian_square(S, c, rq0, rq1, rq2); };
    // the 64-bit sums and means of planes k (buffer n0) and k+1 (n1)
    auto narrow = [&](const uint64_t* n0, const uint64_t* n1, bool two) {
        const uint64_t uA = cA + c0A, uB = cB + c0B;
        {
            const ulonglong2 ym = *(const ulonglong2*)(n0 + own - kSW), yp = *(const ulonglong2*)(n0 + own + kSW);
            const uint64_t SA = uA + cB + n0[own - 1] + ym.x + yp.x + zmA;
            const uint64_t SB = uB + cA + n0[own + 2] + ym.y + yp.y + zmB;
            if constexpr (RM != 2) {
                const double2 o = make_double2(nframe::mean7(SA, nscale), nframe::mean7(SB, nscale));
                if (k1) {
                    *(double2*)out = o;
                    lzm = min(lzm, min(clz32((uint32_t)(SA >> 32)), clz32((uint32_t)(SB >> 32))));
                }
            }
            if constexpr (RM != 0) {
                if (k1) {
                    lsq(SA, cA);
                    lsq(SB, cB);
                }
            }
        }
        if (two) {
            const ulonglong2 ym = *(const ulonglong2*)(n1 + own - kSW), yp = *(const ulonglong2*)(n1 + own + kSW);
            const uint64_t SA = uA + c0B + n1[own - 1] + ym.x + yp.x + c1A;
            const uint64_t SB = uB + c0A + n1[own + 2] + ym.y + yp.y + c1B;
            if constexpr (RM != 2) {
                const double2 o = make_double2(nframe::mean7(SA, nscale), nframe::mean7(SB, nscale));
                if (k1) {
                    *(double2*)(out + plane) = o;
                    lzm = min(lzm, min(clz32((uint32_t)(SA >> 32)), clz32((uint32_t)(SB >> 32))));
                }
            }
            if constexpr (RM != 0) {
                if (k1) {
                    lsq(SA, c0A);
                    lsq(SB, c0B);
                }
            }
        }
    };
    auto advance = [&](bool two) {
        out += 2 * plane;
        zmA = c0A;
        zmB = c0B;
        gzm = g0;
        cA = c1A;
        cB = c1B;
        gc = g1;
        (void)two;
    };
    // hot step: planes k, k+1 with k + 2 < z1, ring phase S. Returns false,
    // with nothing computed or advanced, when the step needs the 96-bit frame.
    auto hot = [&](auto s_c) -> bool {
        constexpr int S = decltype(s_c)::value;
        constexpr int BS = S / 2;
        copy_c(std::integral_constant<int, S == 0 ? 2 : 0>{});
        cp_async_wait<1>();
        uint64_t* const n0 = nsm + BS * (2 * kPlane);
        uint64_t* const n1 = n0 + kPlane;
        bool ga, gb;
        const double2 v0 = *(const double2*)(rc + (S * kN + tid) * 2);
        const double2 v1 = *(const double2*)(rc + ((S + 1) * kN + tid) * 2);
        c0A = nframe::of(v0.x, elo, ga);
        c0B = nframe::of(v0.y, elo, gb);
        g0 = ga && gb;
        c1A = nframe::of(v1.x, elo, ga);
        c1B = nframe::of(v1.y, elo, gb);
        g1 = ga && gb;
        *(ulonglong2*)(n0 + ownw) = make_ulonglong2(cA, cB);
        *(ulonglong2*)(n1 + ownw) = make_ulonglong2(c0A, c0B);
        bool gh = true;
        if (halo_warp) {
            if constexpr (kSplit) {
                n0[hslot] = nframe::of0(mye[S * kEr], elo, gh);
            } else {
                bool gh1;
                n0[hslot] = nframe::of0(mye[S * kEr], elo, gh);
                n1[hslot] = nframe::of0(mye[(S + 1) * kEr], elo, gh1);
                gh = gh && gh1;
            }
        }
        const bool bad = !nok || (k1 && !(gzm && gc && g0 && g1)) || (hv && !gh);
        if (__syncthreads_or(bad)) return false;
        narrow(n0, n1, true);
        advance(true);
        return true;
    };
    int k = z0, ph = 0;  // the next step computes plane k (and k+1) from ring slots ph, ph + 1
    // generic step at (k, ph); with `resume` the copies, conversions and
    // stores were made by a hot step that found a value outside the 64-bit
    // frame, and only its computation remains
    auto generic = [&](bool resume) {
        const int S = ph;
        const bool two = k + 1 < z1;           // planes k and k+1
        const bool zfirst = !two;              // plane k+1 is z1
        const bool zsecond = two && k + 2 >= z1;  // plane k+2 is z1
        uint64_t* const n0 = nsm + (S >> 1) * (2 * kPlane);
        uint64_t* const n1 = n0 + kPlane;
        bool fall = true;
        if (!resume) {
            copy_r(S == 0 ? 2 : 0, k + 2);
            cp_async_wait<1>();
            const double2 zh = *(const double2*)(rc + (RD * kN + tid) * 2);
            const double2 v0 = zfirst ? zh : *(const double2*)(rc + (S * kN + tid) * 2);
            const double2 v1 = zsecond ? zh : *(const double2*)(rc + ((S + 1) * kN + tid) * 2);
            // plane z1 is only ever a z neighbour and may be zero; every other
            // plane becomes a cell's own value and must not be
            bool ga, gb;
            c0A = nframe::of0(v0.x, elo, ga);
            c0B = nframe::of0(v0.y, elo, gb);
            g0 = ga && gb && (zfirst || (c0A != 0u && c0B != 0u));
            c1A = c1B = 0u;
            g1 = true;
            if (two) {
                c1A = nframe::of0(v1.x, elo, ga);
                c1B = nframe::of0(v1.y, elo, gb);
                g1 = ga && gb && (zsecond || (c1A != 0u && c1B != 0u));
            }
            *(ulonglong2*)(n0 + ownw) = make_ulonglong2(cA, cB);
            if (two) *(ulonglong2*)(n1 + ownw) = make_ulonglong2(c0A, c0B);
            bool gh = true;
            if (halo_warp) {
                if constexpr (kSplit) {
                    if (two || hq == 0) n0[hslot] = nframe::of0(mye[S * kEr], elo, gh);
                } else {
                    bool gh1;
                    n0[hslot] = nframe::of0(mye[S * kEr], elo, gh);
                    if (two) {
                        n1[hslot] = nframe::of0(mye[(S + 1) * kEr], elo, gh1);
                        gh = gh && gh1;
                    }
                }
            }
            const bool bad = !nok || (k1 && !(gzm && gc && g0 && g1)) || (hv && !gh);
            if (!__syncthreads_or(bad)) {
                narrow(n0, n1, two);
                fall = false;
            }
        }
        if constexpr (RM != 0) rbad |= fall;
        if (RM != 2 && fall) {
            // the step in the 96-bit frame from the raw values: plane k in the
            // first pair of 64-bit planes, plane k+1 in the second (every
            // thread has passed the step's barrier, so no 64-bit plane is read
            // any more)
            W* const A = (W*)nsm;
            W* const B = A + kPlane;
            W fc0{}, fc1{}, fz0{}, fz1{}, f00{}, f01{}, f10{}, f11{};
            if (k1) {
                const T* pk = osrc - (RD + 1) * plane;  // osrc is at plane k + RD + 1
                // L1-allocating loads, like the ring's cp.async.ca copies, which
                // brought these lines in: in the persistent form the dependency
                // acquire and the barrier before the tile order them after the
                // writers' releases
                const double2 c = *(const double2*)pk;
                const double2 zm = *(const double2*)((k == z0 && z0 == 0) ? z_pair_source<PULL>(pool, desc, d, p, x, y, 4)
                                                                          : pk - plane);
                const double2 zh = *(const double2*)(rc + (RD * kN + tid) * 2);
                const double2 a = zfirst ? zh : *(const double2*)(rc + (S * kN + tid) * 2);
                const double2 bb = zsecond ? zh : *(const double2*)(rc + ((S + 1) * kN + tid) * 2);
                fc0 = frame::of(c.x, eref);
                fc1 = frame::of(c.y, eref);
                fz0 = frame::of(zm.x, eref);
                fz1 = frame::of(zm.y, eref);
                f00 = frame::of(a.x, eref);
                f01 = frame::of(a.y, eref);
                if (two) {
                    f10 = frame::of(bb.x, eref);
                    f11 = frame::of(bb.y, eref);
                }
            }
            A[ownw] = fc0;
            A[ownw + 1] = fc1;
            if (two) {
                B[ownw] = f00;
                B[ownw + 1] = f01;
            }
            if (halo_warp) {
                if constexpr (kSplit) {
                    if (two || hq == 0) (hq ? B : A)[hbase] = frame::of(mye[S * kEr], eref);
                } else {
                    A[hbase] = frame::of(mye[S * kEr], eref);
                    if (two) B[hbase] = frame::of(mye[(S + 1) * kEr], eref);
                }
            }
            __syncthreads();
            auto put = [&](const W& c, const W& xm, const W& xp, const W& ym, const W& yp, const W& zm, const W& zp,
                           T* o, int kk, int cell) {
                uint32_t a0, a1, a2;
                double v;
                frame::sum7(c, xm, xp, ym, yp, zm, zp, a0, a1, a2);
                if (frame::mean7_of_sum(a0, a1, a2, eref, v)) {
                    *o = v;
                    lzm = min(lzm, eref - exp_field(v));
                } else {
                    const int i = atomicAdd(&slow->n, 1);
                    if (i < kSlowMax) slow->cell[i] = ((uint32_t)kk << 10) | ((uint32_t)tid << 1) | (uint32_t)cell;
                }
            };
            if (k1) {
                const int o = own;
                put(fc0, A[o - 1], fc1, A[o - kSW], A[o + kSW], fz0, f00, out, k, 0);
                put(fc1, fc0, A[o + 2], A[o + 1 - kSW], A[o + 1 + kSW], fz1, f01, out + 1, k, 1);
                if (two) {
                    put(f00, B[o - 1], f01, B[o - kSW], B[o + kSW], fc0, f10, out + plane, k + 1, 0);
                    put(f01, f00, B[o + 2], B[o + 1 - kSW], B[o + 1 + kSW], fc1, f11, out + plane + 1, k + 1, 1);
                }
            }
            __syncthreads();  // the next step's 64-bit stores overwrite A and B
        }
        advance(two);
        k += two ? 2 : 1;
        ph ^= 2;
    };
    using S0 = std::integral_constant<int, 0>;
    using S2 = std::integral_constant<int, 2>;
    for (;;) {
        bool stop = false;
        if (ph == 0) {
            for (; k + 4 < z1; k += 4) {
                if (!hot(S0{})) {
                    stop = true;
                    break;
                }
                if (!hot(S2{})) {
                    k += 2;
                    ph = 2;
                    stop = true;
                    break;
                }
            }
        }
        if (stop) generic(true);
        // realign the ring phase, or the tile's last planes
        while (k < z1 && (ph != 0 || k + 4 >= z1)) generic(false);
        if (k >= z1) break;
    }
    cp_async_wait<0>();
    if constexpr (RM != 0) {
        ro->q0 = rq0;
        ro->q1 = rq1;
        ro->q2 = rq2;
        ro->bad = rbad;
    }
    if constexpr (RM == 2) {
        __syncthreads();  // the shared memory is free for the caller
        return;
    }
    n2_slow_cells<PULL, CG, TW>(pool, desc, d, b, p, x0, y0, z0, z1, k1, x, y, slow, eref, lzm);
    if (uout) {
        // every output's exponent field is at most eref - (the least count);
        // published with the tile's results (the barrier and fence before the
        // block's completion counter, or the end of the launch)
        const int w = __reduce_min_sync(0xffffffffu, lzm);
        if ((tid & 31) == 0) atomicMax(uout, (uint32_t)max(0, eref - w));
    }
}

// One binary64 work unit (TW x 512/TW columns) of the exact mean: the
// two-column engine for blocks of even x extent, else the single-column
// engine on the unit's two halves.
template <bool PULL, bool CG, int TW>
__device__ __forceinline__ void exact_unit(double* pool, const BlockDesc* desc, const int32_t* frame_e, int b, int p,
                                           int x0, int y0, int z0, int z1, SlowList* slow, const uint32_t* uin,
                                           uint32_t* uout, FrameSources fsrc = {nullptr, -1})
{
    if ((desc[b].ext[0] & 1) == 0) {
        tile_engine_narrow2<PULL, CG, TW>(pool, desc, frame_e, b, p, x0, y0, z0, z1, jac_dyn_sm, slow, uin, uout,
                                          nullptr, fsrc);
    } else {
        // (the single-column form keeps the grid's frame; its units' bounds stay unknown)
        tile_engine_narrow<PULL, CG, kRing<double>, TW>(pool, desc, frame_e, b, p, x0, y0, z0, z1, jac_dyn_sm, slow);
        const int y1 = y0 + kNT<double> / TW;
        if (y1 < desc[b].ext[1]) {
            __syncthreads();
            tile_engine_narrow<PULL, CG, kRing<double>, TW>(pool, desc, frame_e, b, p, x0, y1, z0, z1, jac_dyn_sm,
                                                            slow);
        }
    }
}

// One binary64 work unit of the sequential rule: the single-plane engine on
// the unit's two halves (TW x 256/TW columns each).
template <bool PULL, bool CG, int TW>
__device__ __forceinline__ void seq_unit(double* pool, const BlockDesc* desc, int b, int p, int x0, int y0, int z0,
                                         int z1)
{
    tile_engine<double, OP_SEQ, PULL, CG, kRing<double>, TW>(pool, desc, b, p, x0, y0, z0, z1, jac_dyn_sm);
    const int y1 = y0 + kNT<double> / TW;
    if (y1 < desc[b].ext[1]) {
        __syncthreads();
        tile_engine<double, OP_SEQ, PULL, CG, kRing<double>, TW>(pool, desc, b, p, x0, y1, z0, z1, jac_dyn_sm);
    }
}

// Dynamic shared memory of the update kernels for op OP.
template <typename T, int OP, int TW>
__host__ __device__ constexpr int kernel_bytes()
{
    if constexpr (OP == OP_EXACT) {
        constexpr int a = n2_engine_bytes<TW>(), b = narrow_engine_bytes<TW, kRing<T>>();
        return a > b ? a : b;
    } else {
        return engine_bytes<T, OP, TW, kRing<T>>();
    }
}

// ------------------------------------------------------- ring engine (SEQ)
// The floating-point rule needs no conversion, so the prefetch ring itself is
// the exchange plane: ring slot q holds the whole (TW + 2) x (TY + 2) tile
// plane q (interior columns, the halo ring, halo cells inside the tile).
// Every thread copies its stream(s) ahead with cp.async straight into the
// slot; after a wait and one barrier per batch of kB planes, the cells of the
// batch read their x/y neighbours from the slot and carry the z neighbours in
// registers (the value above the unit's last plane is loaded once).
constexpr int kSeqBatch = 4;
template <typename T>
constexpr int kSeqAhead = sizeof(T) == 4 ? 3 : 1;  // batches in flight beyond the next
template <typename T>
constexpr int kSeqRing = (kSeqAhead<T> + 3) * kSeqBatch;  // planes in the ring

template <int TW>
__host__ __device__ constexpr int seq_plane()
{
    return (kNT<float> / TW + 2) * (TW + 2) + 1;  // + one slot written by threads without a halo slot
}

template <typename T, int TW>
__host__ __device__ constexpr int seq_engine_bytes()
{
    return kSeqRing<T> * seq_plane<TW>() * (int)sizeof(T);
}

template <typename T, bool PULL, bool CG, int TW>
__device__ void tile_engine_ring(T* __restrict__ pool, const BlockDesc* __restrict__ desc, int b, int p, int x0,
                                 int y0, int z0, int z1, unsigned char* smraw)
{
    constexpr int kB = kSeqBatch, kP = kSeqAhead<T>, RD = kSeqRing<T>;
    constexpr int kTX = TW, kSW = TW + 2, kPl = seq_plane<TW>();
    constexpr uint32_t kPlB = kPl * sizeof(T);
    T* const ring = (T*)smraw;  // [RD][kPl]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const int x = x0 + tx, y = y0 + ty;
    const int64_t plane = d.plane;

    // own stream: planes z0 .. z1-1 of the column (kind 1) or of the halo cell
    // inside the tile (kind 2); q_end = z0 for threads with no stream
    const bool k1 = x < bx && y < by;
    const bool k2 = (x == bx && y < by) || (y == by && x < bx);
    const T* op = pool;
    int64_t ostr = 0;
    int oend = z0;
    T zm = T(0), zhiv = T(0);
    T* out = pool;
    if (k1) {
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        op = col + z0 * plane;
        ostr = plane;
        oend = z1;
        zm = ldv<T, CG>(z0 == 0 ? z_source<T, PULL>(pool, desc, d, p, x, y, 4) : col + (z0 - 1) * plane);
        zhiv = ldv<T, CG>(z1 == bz ? z_source<T, PULL>(pool, desc, d, p, x, y, 5) : col + z1 * plane);
        out = pool + cell_index<T>(d, p ^ 1, x, y, z0);
    } else if (k2) {
        const Src<T> s = xy_source<T, PULL>(pool, desc, d, p, x, y);
        op = s.p + z0 * s.stride;
        ostr = s.stride;
        oend = z1;
    }
    const HaloSlot<T> hs = halo_slot<T, PULL, TW>(pool, desc, d, p, x0, y0, z0, tid);
    const bool hv = hs.er >= 0;
    const T* hp = hs.p;
    const int64_t hstr = hs.stride;
    const int hend = hv ? z1 : z0;
    const int own = (ty + 1) * kSW + tx + 1;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t own_s = ring_s + own * sizeof(T);
    const uint32_t halo_s = ring_s + (hv ? hs.er * kSW + hs.ec : kPl - 1) * sizeof(T);

    // Copy batch m holds planes z0 + m kB .. z0 + m kB + kB - 1 in ring slots
    // (m kB + i) % RD. Batch j of the update computes planes k0 .. k0+kB-1
    // (k0 = z0 + j kB) and reads planes k0 .. k0+kB: copy batches up to j + 1
    // must have landed. It first issues batch j + kP + 1, whose slots last
    // held planes read two barriers ago. The z loop runs a whole ring turn
    // (RD / kB batches) per pass, so every slot index is a constant; passes
    // whose planes and copies all lie inside the range skip the range checks.
    constexpr int kNB = RD / kB;
    static_assert(RD % kB == 0, "ring of whole batches");
    const bool halo_warp = (tid & ~31) < ring_extra<T, TW>();  // warp-uniform
    const bool own_on = oend > z0, halo_on = hend > z0;
    int cq = z0;  // the next plane to copy
    // copy batch into slots sb * kB .. sb * kB + kB - 1
    auto copy_batch = [&](auto full_c, auto sb_c) {
        constexpr bool FULL = decltype(full_c)::value;
        constexpr int sb = decltype(sb_c)::value;
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const uint32_t so = (uint32_t)((sb * kB + i) * kPlB);
            cp_async_if<sizeof(T)>(own_s + so, op, FULL ? own_on : cq + i < oend);
            op += ostr;
        }
        if (halo_warp) {
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const uint32_t so = (uint32_t)((sb * kB + i) * kPlB);
                cp_async_if<sizeof(T)>(halo_s + so, hp, FULL ? halo_on : cq + i < hend);
                hp += hstr;
            }
        }
        cq += kB;
        cp_async_commit();
    };
    // prologue: batches 0 .. kP
    [&]<int... M>(std::integer_sequence<int, M...>) {
        (copy_batch(std::false_type{}, std::integral_constant<int, M>{}), ...);
    }(std::make_integer_sequence<int, kP + 1>{});

    const T* const rd = ring + own;  // plane in slot q: rd[q * kPl]
    T c;
    cp_async_wait<kP>();
    __syncthreads();
    c = rd[0];
    // one batch: j-th of the pass starting at kb
    auto batch = [&](auto full_c, auto bi_c, int kb) {
        constexpr bool FULL = decltype(full_c)::value;
        constexpr int bi = decltype(bi_c)::value;
        const int k0 = kb + bi * kB;
        copy_batch(full_c, std::integral_constant<int, (bi + kP + 1) % kNB>{});
        cp_async_wait<kP>();
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int k = k0 + i;
            if (FULL || k < z1) {
                const int q = bi * kB + i, qn = (q + 1) % RD;
                const T* pl = rd + q * kPl;
                const T zp = (FULL || k + 1 < z1) ? rd[qn * kPl] : zhiv;
                const T o = mean7<T, 0>(c, pl[-1], pl[1], pl[-kSW], pl[kSW], zm, zp);
                if (k1) *out = o;
                out += plane;
                zm = c;
                c = zp;
            }
        }
    };
    auto pass = [&](auto full_c, int kb) {
        [&]<int... J>(std::integer_sequence<int, J...>) {
            (batch(full_c, std::integral_constant<int, J>{}, kb), ...);
        }(std::make_integer_sequence<int, kNB>{});
    };
    int kb = z0;
    // a full pass computes planes kb .. kb+RD-1 (each with a plane above it in
    // the range) and copies planes up to kb + RD + (kP + 1) kB - 1
    for (; kb + RD + (kP + 1) * kB <= z1; kb += RD) pass(std::true_type{}, kb);
    for (; kb < z1; kb += RD) pass(std::false_type{}, kb);
    cp_async_wait<0>();
    __syncthreads();  // the ring is free for the next unit
}

// ------------------------------------------- two-column ring engine (binary32)
// The ring engine with each thread owning an x-adjacent pair of columns:
// 8-byte copies and loads for the pair, 4-byte loads for its two outer x
// neighbours, so a cell costs half the shared-memory instructions. A tile is
// TW x (1024 / TW) cells. Plane rows are laid out [pad, left halo, TW
// interior, right halo, pad] so every pair sits on an 8-byte boundary. Used
// when the block's x extent is even (pairs never straddle the block edge).
constexpr int kR2Batch = 4, kR2Ahead = 2;
constexpr int kR2Ring = (kR2Ahead + 3) * kR2Batch;

template <int TW>
__host__ __device__ constexpr int ring2_rows()
{
    return 2 * kNT<float> / TW;
}

template <int TW>
__host__ __device__ constexpr int ring2_plane()
{
    return (ring2_rows<TW>() + 2) * (TW + 4) + 2;  // + one pair written by threads without a halo slot
}

template <int TW>
__host__ __device__ constexpr int ring2_bytes()
{
    return kR2Ring * ring2_plane<TW>() * (int)sizeof(float);
}

// Where a pair of x-adjacent cells (x, x+1) lives along z (x even, both in
// the block or both in one neighbouring block); a Dirichlet constant is read
// from its duplicated form.
__device__ __forceinline__ Src<float> pair_source(const float* pool, const BlockDesc* desc, const BlockDesc& d, int p,
                                                  int x, int y)
{
    Src<float> s = xy_source<float, true>(pool, desc, d, p, x, y);
    if (s.stride == 0) s.p = d.bcf2[s.p - d.bcf];
    return s;
}

__device__ __forceinline__ float2 ld2(const float* p) { return *(const float2*)p; }
__device__ __forceinline__ float2 ldcg2(const float* p) { return __ldcg((const float2*)p); }

// What the engine's residual modes return per thread: the exact sums of the
// split Laplacian terms of its interior cells, and whether a value it read
// lies outside the split's exact range (or the grid's frame is out of range).
struct R32Out {
    r32::Acc acc;
    bool bad;
};

// RM (residual mode): 0 the update only; 1 the update and, from the same
// values, the residual terms of the grid it reads; 2 the residual terms only.
template <bool CG, int TW, int RM = 0>
__device__ __forceinline__ void tile_engine_ring2(float* __restrict__ pool, const BlockDesc* __restrict__ desc, int b,
                                                  int p, int x0, int y0, int z0, int z1, unsigned char* smraw,
                                                  const int32_t* frame_e = nullptr, R32Out* ro = nullptr)
{
    using T = float;
    constexpr int kB = kR2Batch, kP = kR2Ahead, RD = kR2Ring, kNB = RD / kB;
    constexpr int kTPR = TW / 2, kTY = ring2_rows<TW>(), kSW = TW + 4, kPl = ring2_plane<TW>();
    constexpr uint32_t kPlB = kPl * sizeof(T);
    static_assert(RD % kB == 0, "ring of whole batches");
    T* const ring = (T*)smraw;  // [RD][kPl]
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int tid = threadIdx.x, tx = tid % kTPR, ty = tid / kTPR;
    const int x = x0 + 2 * tx, y = y0 + ty;  // the pair (x, y), (x + 1, y)
    const int64_t plane = d.plane;
    auto ldp = [&](const T* q) { return CG ? ldcg2(q) : ld2(q); };

    // own stream: an interior pair (k1); a pair of the y-halo row inside the
    // tile (k2p, 8-byte copies); the x-halo column inside the tile (k2s, the
    // pair's first cell, 4-byte copies)
    const bool k1 = x < bx && y < by;
    const bool k2p = y == by && x < bx;
    const bool k2s = x == bx && y < by;
    const T* op = pool;
    int64_t ostr = 0;
    float2 zm = make_float2(0.f, 0.f), zhiv = zm;
    T* out = pool;
    if (k1) {
        const T* col = pool + cell_index<T>(d, p, x, y, 0);
        op = col + z0 * plane;
        ostr = plane;
        out = pool + cell_index<T>(d, p ^ 1, x, y, z0);
        if (z0 > 0) zm = ldp(col + (z0 - 1) * plane);
        else if (d.nbr[4] < 0) zm = make_float2(d.bcf[4], d.bcf[4]);
        else {
            const BlockDesc& n = desc[d.nbr[4]];
            zm = ldp(pool + cell_index<T>(n, p, x, y, n.ext[2] - 1));
        }
        if (z1 < bz) zhiv = ldp(col + z1 * plane);
        else if (d.nbr[5] < 0) zhiv = make_float2(d.bcf[5], d.bcf[5]);
        else zhiv = ldp(pool + cell_index<T>(desc[d.nbr[5]], p, x, y, 0));
    } else if (k2p) {
        const Src<T> s = pair_source(pool, desc, d, p, x, y);
        op = s.p + z0 * s.stride;
        ostr = s.stride;
    } else if (k2s) {
        const Src<T> s = xy_source<T, true>(pool, desc, d, p, x, y);
        op = s.p + z0 * s.stride;
        ostr = s.stride;
    }
    const bool own8 = k1 || k2p, own4 = k2s;
    const int own = (ty + 1) * kSW + 2 * tx + 2;

    // halo-ring slots: top and bottom rows as pairs (8 bytes), left and right
    // columns as single cells (4 bytes); threads without one use the dummy pair
    bool h8 = false, h4 = false;
    int hslot = kPl - 2;
    const T* hp = pool;
    int64_t hstr = 0;
    if (tid < 2 * kTPR + 2 * kTY) {
        int hx, hy, slot;
        bool pair, valid;
        if (tid < kTPR) {
            hx = x0 + 2 * tid;
            hy = y0 - 1;
            slot = 2 * tid + 2;
            pair = true;
            valid = hx < bx;
        } else if (tid < 2 * kTPR) {
            const int c = tid - kTPR;
            hx = x0 + 2 * c;
            hy = y0 + kTY;
            slot = (kTY + 1) * kSW + 2 * c + 2;
            pair = true;
            valid = hx < bx && hy <= by;
        } else if (tid < 2 * kTPR + kTY) {
            const int r = tid - 2 * kTPR;
            hx = x0 - 1;
            hy = y0 + r;
            slot = (r + 1) * kSW + 1;
            pair = false;
            valid = hy < by;
        } else {
            const int r = tid - 2 * kTPR - kTY;
            hx = x0 + TW;
            hy = y0 + r;
            slot = (r + 1) * kSW + TW + 2;
            pair = false;
            valid = hy < by && hx <= bx;
        }
        if (valid) {
            const Src<T> hs = pair ? pair_source(pool, desc, d, p, hx, hy) : xy_source<T, true>(pool, desc, d, p, hx, hy);
            hp = hs.p + z0 * hs.stride;
            hstr = hs.stride;
            hslot = slot;
            h8 = pair;
            h4 = !pair;
        }
    }
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t own_s = ring_s + own * sizeof(T);
    const uint32_t halo_s = ring_s + hslot * sizeof(T);
    const bool halo_warp = (tid & ~31) < 2 * kTPR + 2 * kTY;  // warp-uniform

    int cq = z0;  // the next plane to copy
    // copy batch into ring slots sb .. sb + kB - 1 (sb a multiple of kB)
    auto copy_batch = [&](auto full_c, int sb) {
        constexpr bool FULL = decltype(full_c)::value;
        const uint32_t so = (uint32_t)sb * kPlB;
        const uint32_t od = own_s + so, hd = halo_s + so;
        [&]<int... I>(std::integer_sequence<int, I...>) {
            ((cp_async_if_off<8, I * (int)kPlB>(od, op + I * ostr, own8 && (FULL || cq + I < z1)),
              cp_async_if_off<4, I * (int)kPlB>(od, op + I * ostr, own4 && (FULL || cq + I < z1))),
             ...);
        }(std::make_integer_sequence<int, kB>{});
        op += kB * ostr;
        if (halo_warp) {
            [&]<int... I>(std::integer_sequence<int, I...>) {
                ((cp_async_if_off<8, I * (int)kPlB>(hd, hp + I * hstr, h8 && (FULL || cq + I < z1)),
                  cp_async_if_off<4, I * (int)kPlB>(hd, hp + I * hstr, h4 && (FULL || cq + I < z1))),
                 ...);
            }(std::make_integer_sequence<int, kB>{});
            hp += kB * hstr;
        }
        cq += kB;
        cp_async_commit();
    };
#pragma unroll
    for (int m = 0; m <= kP; ++m) copy_batch(std::false_type{}, m * kB);

    const T* const rd = ring + own;  // the pair of the plane in slot q: rd[q * kPl]
    cp_async_wait<kP>();
    __syncthreads();
    float2 c = ld2(rd);
    // residual modes: the split constants of the block's grid, the own pair's
    // splits at planes k (rc*) and k - 1 (rz*), and the exact sums. Every value
    // a cell reads is checked by one lane at least: its own tile's values by
    // their owners (the pair entering as zp, the first plane, the plane below
    // the range), the x halo by the lanes reading xm0 and xp1, the y halo rows
    // by the warps holding the tile's first and last rows, the row at the
    // block's y edge by its k2p owners.
    [[maybe_unused]] float c1 = 0.f, c2 = 0.f;
    [[maybe_unused]] bool rbad = false;
    [[maybe_unused]] r32::Acc racc{0, 0, 0};
    [[maybe_unused]] r32::Split rc0{}, rc1{}, rz0{}, rz1{};
    [[maybe_unused]] const bool ylo_warp = (tid >> 5) == 0, yhi_warp = (tid >> 5) == kNT<T> / 32 - 1;
    if constexpr (RM != 0) {
        const int E = r32::frame_E(frame_e[d.inst] - 896);
        rbad = !r32::frame_ok(E);
        const int Ec = rbad ? 0 : E;  // finite constants either way
        c1 = r32::c15(Ec + 1);
        c2 = r32::c15(Ec - 22);
        bool eo = false, ez = false;
        rc0 = r32::split(c.x, c1, c2, eo);
        rc1 = r32::split(c.y, c1, c2, eo);
        rz0 = r32::split(zm.x, c1, c2, ez);
        rz1 = r32::split(zm.y, c1, c2, ez);
        rbad |= ((k1 || k2p) && eo) || (k1 && ez);
    }
    // Batch j computes planes k0 .. k0+kB-1 (slots q0 ..) and reads plane
    // k0+kB too; it first issues copy batch j + kP + 1 into slots sb ..
    int q0 = 0, sb = (kP + 1) * kB;
    auto batch = [&](auto full_c, int k0) {
        constexpr bool FULL = decltype(full_c)::value;
        copy_batch(full_c, sb);
        cp_async_wait<kP>();
        __syncthreads();
        const T* const p0 = rd + q0 * kPl;
        const int qe = q0 + kB == RD ? 0 : q0 + kB;  // slot of plane k0 + kB
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int k = k0 + i;
            if (FULL || k < z1) {
                const T* pl = p0 + i * kPl;
                const T* pn = i + 1 < kB ? pl + kPl : rd + qe * kPl;
                const float2 zp = (FULL || k + 1 < z1) ? ld2(pn) : zhiv;
                const float xm0 = pl[-1], xp1 = pl[2];
                const float2 ym = ld2(pl - kSW), yp = ld2(pl + kSW);
                if constexpr (RM != 2) {
                    float s0 = __fadd_rn(c.x, xm0);
                    s0 = __fadd_rn(s0, c.y);
                    s0 = __fadd_rn(s0, ym.x);
                    s0 = __fadd_rn(s0, yp.x);
                    s0 = __fadd_rn(s0, zm.x);
                    s0 = __fadd_rn(s0, zp.x);
                    float s1 = __fadd_rn(c.y, c.x);
                    s1 = __fadd_rn(s1, xp1);
                    s1 = __fadd_rn(s1, ym.y);
                    s1 = __fadd_rn(s1, yp.y);
                    s1 = __fadd_rn(s1, zm.y);
                    s1 = __fadd_rn(s1, zp.y);
                    float2 o = make_float2(div7f_fast(s0), div7f_fast(s1));
                    // the exact small-value path, for the warp only when a lane needs it
                    if (__any_sync(0xffffffffu, k1 && (div7f_needs_exact(s0) || div7f_needs_exact(s1)))) {
                        o.x = div7f(s0);
                        o.y = div7f(s1);
                    }
                    if (k1) *(float2*)out = o;
                }
                if constexpr (RM != 0) {
                    // L of the pair's cells at plane k, in the split words
                    bool eo = false, ex = false, ey = false;
                    const r32::Split n0 = r32::split(zp.x, c1, c2, eo), n1 = r32::split(zp.y, c1, c2, eo);
                    const r32::Split sxm = r32::split(xm0, c1, c2, ex), sxp = r32::split(xp1, c1, c2, ex);
                    r32::Split sym0, sym1, syp0, syp1;
                    if (ylo_warp) {
                        sym0 = r32::split(ym.x, c1, c2, ey);
                        sym1 = r32::split(ym.y, c1, c2, ey);
                    } else {
                        sym0 = r32::split_nc(ym.x, c1, c2);
                        sym1 = r32::split_nc(ym.y, c1, c2);
                    }
                    if (yhi_warp) {
                        syp0 = r32::split(yp.x, c1, c2, ey);
                        syp1 = r32::split(yp.y, c1, c2, ey);
                    } else {
                        syp0 = r32::split_nc(yp.x, c1, c2);
                        syp1 = r32::split_nc(yp.y, c1, c2);
                    }
                    rbad |= ((k1 || k2p) && eo) || (k1 && (ex || ey));
                    const int32_t h0 = r32::lpart(rc0.h, sxm.h, rc1.h, sym0.h, syp0.h, rz0.h, n0.h);
                    const int32_t g0 = r32::lpart(rc0.g, sxm.g, rc1.g, sym0.g, syp0.g, rz0.g, n0.g);
                    const int32_t h1 = r32::lpart(rc1.h, rc0.h, sxp.h, sym1.h, syp1.h, rz1.h, n1.h);
                    const int32_t g1 = r32::lpart(rc1.g, rc0.g, sxp.g, sym1.g, syp1.g, rz1.g, n1.g);
                    if (k1) {
                        r32::add_square(h0, g0, racc);
                        r32::add_square(h1, g1, racc);
                    }
                    rz0 = rc0;
                    rz1 = rc1;
                    rc0 = n0;
                    rc1 = n1;
                }
                out += plane;
                zm = c;
                c = zp;
            }
        }
        q0 = qe;
        sb = sb + kB == RD ? 0 : sb + kB;
    };
    int k0 = z0;
    // a FULL batch: its planes, the plane above them and its copies (up to
    // plane k0 + (kP + 2) kB - 1) all lie inside the range
    for (; k0 + (kP + 2) * kB <= z1; k0 += kB) batch(std::true_type{}, k0);
    for (; k0 < z1; k0 += kB) batch(std::false_type{}, k0);
    cp_async_wait<0>();
    __syncthreads();  // the ring is free for the next unit
    if constexpr (RM != 0) {
        ro->acc = racc;
        ro->bad = rbad;
    }
}

// A binary32 unit (TW x 1024/TW cells): the two-column engine when the
// block's x extent is even, else the scalar ring engine on its two halves.
template <bool CG, int TW>
__device__ __forceinline__ void f32_unit(float* pool, const BlockDesc* desc, int b, int p, int x0, int y0, int z0,
                                         int z1)
{
    if ((desc[b].ext[0] & 1) == 0) {
        tile_engine_ring2<CG, TW>(pool, desc, b, p, x0, y0, z0, z1, jac_dyn_sm);
    } else {
        tile_engine_ring<float, true, CG, TW>(pool, desc, b, p, x0, y0, z0, z1, jac_dyn_sm);
        tile_engine_ring<float, true, CG, TW>(pool, desc, b, p, x0, y0 + kNT<float> / TW, z0, z1, jac_dyn_sm);
    }
}

template <int TW>
__host__ __device__ constexpr int f32_unit_bytes()
{
    return ring2_bytes<TW>() > seq_engine_bytes<float, TW>() ? ring2_bytes<TW>() : seq_engine_bytes<float, TW>();
}

// Work units carry their tile width (16, 32 or 64, chosen per block-width
// class by the autotuner): the unit kernels dispatch on it.
template <typename F>
__device__ __forceinline__ void with_tw(int tw, F&& f)
{
    if (tw == 16) f(std::integral_constant<int, 16>{});
    else if (tw == 64) f(std::integral_constant<int, 64>{});
    else f(std::integral_constant<int, 32>{});
}

template <typename T>
__global__ void __launch_bounds__(kNT<T>, kMinCTAs<T>) k_fused_ring(T* pool, const BlockDesc* desc, const TileUnit* units, int p)
{
    const TileUnit u = units[blockIdx.x];
    with_tw(u.tw, [&](auto tw_c) {
        constexpr int TW = decltype(tw_c)::value;
        f32_unit<false, TW>(pool, desc, u.block, p, u.x0, u.y0, u.z0, u.z1);
    });
}

template <typename T, int OP, int TW>
__global__ void __launch_bounds__(kNT<T>, (kMinCTAsOp<T, OP>)) k_stencil_block(T* pool, const BlockDesc* desc, const int32_t* frame_e,
                                                               int b, int p)
{
    __shared__ SlowList slow;
    if constexpr (OP == OP_EXACT)
        exact_unit<false, false, TW>(pool, desc, frame_e, b, p, blockIdx.x * TW, blockIdx.y * (2 * kNT<T> / TW), 0,
                                     desc[b].ext[2], &slow, nullptr, nullptr);
    else
        tile_engine<T, OP, false, false, kRing<T>, TW>(pool, desc, b, p, blockIdx.x * TW, blockIdx.y * (kNT<T> / TW),
                                                       0, desc[b].ext[2], jac_dyn_sm);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kNT<T>, (kMinCTAsOp<T, OP>)) k_fused_step(T* pool, const BlockDesc* desc, const int32_t* frame_e,
                                                            const TileUnit* units, int p, uint32_t* uexp, int ucap,
                                                            const int32_t* fs)
{
    __shared__ SlowList slow;
    const TileUnit u = units[blockIdx.x];
    with_tw(u.tw, [&](auto tw_c) {
        constexpr int TW = decltype(tw_c)::value;
        if constexpr (OP == OP_EXACT)
            exact_unit<true, false, TW>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1, &slow,
                                        uexp + (int64_t)p * ucap, uexp + (int64_t)(p ^ 1) * ucap + blockIdx.x,
                                        frame_sources(fs, u));
        else
            seq_unit<true, false, TW>(pool, desc, u.block, p, u.x0, u.y0, u.z0, u.z1);
    });
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
template <typename T, int OP, bool RING, int MINB = kMinCTAsOp<T, OP>>
__global__ void __launch_bounds__(kNT<T>, MINB)
    k_persistent(T* pool, const BlockDesc* desc, const int32_t* frame_e, const TileUnit* units, int nunits, int p0,
                 int64_t n_iters, uint32_t* done, unsigned long long* work, DeviceStatus* st, int64_t wait_ns,
                 int hold_block, int64_t hold_after, uint32_t* uexp, int ucap, const int32_t* fs)
{
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
        with_tw(u.tw, [&](auto tw_c) {
            constexpr int TW = decltype(tw_c)::value;
            if constexpr (RING) {
                // L1-allocating copies are safe here: the acquire and the
                // barrier above order them after the neighbours' releases
                f32_unit<true, TW>(pool, desc, u.block, (p0 + t) & 1, u.x0, u.y0, u.z0, u.z1);
            } else if constexpr (OP == OP_EXACT) {
                const int pt = (p0 + t) & 1;
                exact_unit<true, true, TW>(pool, desc, frame_e, u.block, pt, u.x0, u.y0, u.z0, u.z1, &slow,
                                           uexp + (int64_t)pt * ucap, uexp + (int64_t)(pt ^ 1) * ucap + w % nunits,
                                           frame_sources(fs, u));
            } else {
                seq_unit<true, true, TW>(pool, desc, u.block, (p0 + t) & 1, u.x0, u.y0, u.z0, u.z1);
            }
        });
        __syncthreads();
        if (tid == 0 && !(u.block == hold_block && t >= hold_after)) {
            __threadfence();
            atomicAdd(done + u.block, 1u);
        }
    }
}

// ------------------------------------------------------------ residual
// The residual from the two-column engines' residual modes: per work unit
// the exact sum of L^2 (binary32: split words, 128-bit combination; binary64:
// the 64-bit frame's S - 7c, 192-bit squares), rounded once to binary64.
// Units these cannot take (odd x extent, a value outside the exact range, a
// frame out of range) take the two-plane engine (tile_engine_pair's residual
// ops), whose per-unit partial is rounded per thread and summed by a fixed
// tree. The partials are summed by the last unit to finish in a fixed order,
// so the grid's rho is the same bits in every form that produces it.

// partials[unit] = part (thread 0's); with `out` set, the last unit to
// finish (a fence, then an atomic count) writes sqrt of the sum of the
// partials there (256 strided sums in unit order, then a fixed tree) and
// clears *count, which is zero at every launch.
__device__ void finish_residual(double part, double* partials, int nunits, unsigned* count, double* out, int* s_last)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        partials[blockIdx.x] = part;
        if (out) {
            __threadfence();
            *s_last = atomicAdd(count, 1u) == (unsigned)(nunits - 1);
        }
    }
    if (!out) return;
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    double* const red = (double*)jac_dyn_sm;
    if (tid < 256) {
        double acc = 0.0;
        for (int i = tid; i < nunits; i += 256) acc = acc + __ldcg(partials + i);
        red[tid] = acc;
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    if (tid == 0) {
        out[0] = sqrt(red[0]);
        *count = 0u;
    }
}

// The unit's partial from the threads' exact sums (valid in thread 0).
__device__ double r32_unit_partial(const r32::Acc& a, int E, unsigned char* smraw)
{
    uint64_t lo, hi;
    r32::combine(a, lo, hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t ol = __shfl_down_sync(0xffffffffu, lo, o), oh = __shfl_down_sync(0xffffffffu, hi, o);
        const uint64_t nl = lo + ol;
        hi += oh + (nl < ol ? 1u : 0u);
        lo = nl;
    }
    uint64_t* const w = (uint64_t*)smraw;  // [warps][2]
    const int tid = threadIdx.x;
    if ((tid & 31) == 0) {
        w[2 * (tid >> 5)] = lo;
        w[2 * (tid >> 5) + 1] = hi;
    }
    __syncthreads();
    double part = 0.0;
    if (tid == 0) {
        uint64_t sl = 0u, sh = 0u;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            const uint64_t nl = sl + w[2 * i];
            sh += w[2 * i + 1] + (nl < w[2 * i] ? 1u : 0u);
            sl = nl;
        }
        part = frame::u192_to_double_scaled(sl, sh, 0u, 2 * E - 90);
    }
    __syncthreads();
    return part;
}

// The two-plane engine's partial of a unit (valid in thread 0): the two
// engine tiles, then a fixed tree over the threads (binary32 grids: L^2
// summed exactly per thread in a 64-bit frame; binary64: L rounded once,
// fused multiply-adds).
template <typename T, int TW>
__device__ __noinline__ double res_fallback_partial(T* pool, const BlockDesc* desc, const int32_t* frame_e, int b,
                                                    int p, int x0, int y0, int z0, int z1, SlowList* slow)
{
    constexpr int OPR = sizeof(T) == 4 ? OP_RES32 : OP_RES;
    double acc = tile_engine_pair<T, OPR, true, false, kRingRes, TW>(pool, desc, frame_e, b, p, x0, y0, z0, z1,
                                                                     jac_dyn_sm, slow);
    __syncthreads();
    acc += tile_engine_pair<T, OPR, true, false, kRingRes, TW>(pool, desc, frame_e, b, p, x0, y0 + kNT<T> / TW, z0,
                                                               z1, jac_dyn_sm, slow);
    __syncthreads();
    double* const red = (double*)jac_dyn_sm;
    const int tid = threadIdx.x;
    red[tid] = acc;
    __syncthreads();
    for (int s = kNT<T> / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = red[tid] + red[tid + s];
        __syncthreads();
    }
    const double part = red[0];
    __syncthreads();
    return part;
}

// RM 1: one binary32 update iteration (as k_fused_ring) that also returns the
// residual of the grid it reads; RM 2: the residual only. partials[unit] gets
// the unit's partial; with `out` set, the last unit to finish writes
// sqrt(sum of partials) there and clears *count (zero at every launch).
template <int RM>
__global__ void __launch_bounds__(kNT<float>, kMinCTAs<float>)
    k_ring_residual(float* pool, const BlockDesc* desc, const int32_t* frame_e, const TileUnit* units, int nunits,
                    int p, double* partials, unsigned* count, double* out)
{
    __shared__ SlowList slow;
    __shared__ int s_last;
    const TileUnit u = units[blockIdx.x];
    const BlockDesc& d = desc[u.block];
    double part = 0.0;
    with_tw(u.tw, [&](auto tw_c) {
        constexpr int TW = decltype(tw_c)::value;
        bool fall = true;
        if ((d.ext[0] & 1) == 0) {
            R32Out ro;
            tile_engine_ring2<false, TW, RM>(pool, desc, u.block, p, u.x0, u.y0, u.z0, u.z1, jac_dyn_sm, frame_e,
                                             &ro);
            fall = __syncthreads_or(ro.bad);
            if (!fall) part = r32_unit_partial(ro.acc, r32::frame_E(frame_e[d.inst] - 896), jac_dyn_sm);
        } else if constexpr (RM == 1) {
            tile_engine_ring<float, true, false, TW>(pool, desc, u.block, p, u.x0, u.y0, u.z0, u.z1, jac_dyn_sm);
            tile_engine_ring<float, true, false, TW>(pool, desc, u.block, p, u.x0, u.y0 + kNT<float> / TW, u.z0,
                                                     u.z1, jac_dyn_sm);
        }
        if (fall)
            part = res_fallback_partial<float, TW>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1, &slow);
    });
    finish_residual(part, partials, nunits, count, out, &s_last);
}

// The exact partial of a binary64 unit from the threads' 192-bit sums of
// L^2 (units of 2^scale), rounded once (valid in thread 0).
__device__ double r64_unit_partial(const R64Out& r, int scale, unsigned char* smraw)
{
    uint64_t a0 = r.q0, a1 = r.q1, a2 = r.q2;
    auto add3 = [](uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t y0, uint64_t y1, uint64_t y2) {
        const uint64_t s0 = x0 + y0;
        const uint64_t c0 = s0 < y0 ? 1u : 0u;
        const uint64_t t1 = x1 + y1;
        const uint64_t c1 = t1 < y1 ? 1u : 0u;
        const uint64_t s1 = t1 + c0;
        const uint64_t c2 = s1 < t1 ? 1u : 0u;
        x0 = s0;
        x1 = s1;
        x2 += y2 + c1 + c2;
    };
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t b0 = __shfl_down_sync(0xffffffffu, a0, o), b1 = __shfl_down_sync(0xffffffffu, a1, o),
                       b2 = __shfl_down_sync(0xffffffffu, a2, o);
        add3(a0, a1, a2, b0, b1, b2);
    }
    uint64_t* const w = (uint64_t*)smraw;  // [warps][3]
    const int tid = threadIdx.x;
    __syncthreads();
    if ((tid & 31) == 0) {
        w[3 * (tid >> 5)] = a0;
        w[3 * (tid >> 5) + 1] = a1;
        w[3 * (tid >> 5) + 2] = a2;
    }
    __syncthreads();
    double part = 0.0;
    if (tid == 0) {
        uint64_t s0 = 0u, s1 = 0u, s2 = 0u;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) add3(s0, s1, s2, w[3 * i], w[3 * i + 1], w[3 * i + 2]);
        part = frame::u192_to_double_scaled(s0, s1, s2, scale);
    }
    __syncthreads();
    return part;
}

// RM 1: one binary64 iteration of the correctly rounded mean (the bits of
// k_fused_step, which it replaces, unit bounds included) that also returns
// the residual of the grid it reads; RM 2: the residual only. The 64-bit
// frame is the grid's: a unit with a step outside it, of odd x extent, or
// whose sum of squares could leave the normal range (scale outside
// [-1000, 800]) takes the two-plane engine. Partials and the grid's sum as in
// k_ring_residual.
template <int RM>
__global__ void __launch_bounds__(kNT<double>, 2)
    k_narrow_residual(double* pool, const BlockDesc* desc, const int32_t* frame_e, const TileUnit* units, int nunits,
                      int p, uint32_t* uexp, int ucap, double* partials, unsigned* count, double* out)
{
    __shared__ SlowList slow;
    __shared__ int s_last;
    const TileUnit u = units[blockIdx.x];
    const BlockDesc& d = desc[u.block];
    double part = 0.0;
    with_tw(u.tw, [&](auto tw_c) {
        constexpr int TW = decltype(tw_c)::value;
        uint32_t* const uout = RM == 1 ? uexp + (int64_t)(p ^ 1) * ucap + blockIdx.x : nullptr;
        bool fall = true;
        if ((d.ext[0] & 1) == 0) {
            R64Out ro;
            tile_engine_narrow2<true, false, TW, RM>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1,
                                                     jac_dyn_sm, &slow, nullptr, uout, &ro);
            const int scale = 2 * (frame_e[d.inst] + 1 - 1084);
            fall = __syncthreads_or(ro.bad) || scale < -1000 || scale > 800;
            if (!fall) part = r64_unit_partial(ro, scale, jac_dyn_sm);
        } else if constexpr (RM == 1) {
            exact_unit<true, false, TW>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1, &slow, nullptr,
                                        uout);
            __syncthreads();
        }
        if (fall)
            part = res_fallback_partial<double, TW>(pool, desc, frame_e, u.block, p, u.x0, u.y0, u.z0, u.z1, &slow);
    });
    finish_residual(part, partials, nunits, count, out, &s_last);
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


// The interior/exterior split of the update (the manual overlap of Section
// II-A, Fig. 1): the interior region (cells 1 .. b-2 on every axis) reads
// only the block's own values, so it can run while the halos are exchanged;
// the exterior region (the outermost layer of cells) reads the ghost layer
// and runs after the unpack. One thread per (x, y) column marching in z, the
// z neighbours carried in registers, the per-cell mean of the context's rule.
template <typename T, int OP>
__device__ __forceinline__ T region_mean(T c, T xm, T xp, T ym, T yp, T zm, T zp)
{
    if constexpr (OP == OP_EXACT) return (T)mean7_exact((double)c, (double)xm, (double)xp, (double)ym, (double)yp,
                                                        (double)zm, (double)zp);
    else return mean7<T, 0>(c, xm, xp, ym, yp, zm, zp);
}

template <typename T, int OP>
__global__ void k_update_region(T* pool, const BlockDesc* desc, int b, int p, int exterior)
{
    const BlockDesc& d = desc[b];
    const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= bx || y >= by) return;
    const bool ring = x == 0 || y == 0 || x == bx - 1 || y == by - 1;
    int k0, k1, kstep;
    if (!exterior) {
        if (ring) return;
        k0 = 1;
        k1 = bz - 1;  // planes 1 .. bz-2
        kstep = 1;
    } else if (ring) {
        k0 = 0;
        k1 = bz;
        kstep = 1;
    } else {
        k0 = 0;  // planes 0 and bz-1 of an inner column
        k1 = bz;
        kstep = bz > 1 ? bz - 1 : 1;
    }
    auto at = [&](int xx, int yy, int kk) { return load_cell<T, false, false>(pool, desc, d, p, xx, yy, kk); };
    for (int k = k0; k < k1; k += kstep) {
        const T o = region_mean<T, OP>(at(x, y, k), at(x - 1, y, k), at(x + 1, y, k), at(x, y - 1, k),
                                        at(x, y + 1, k), at(x, y, k - 1), at(x, y, k + 1));
        pool[cell_index<T>(d, p ^ 1, x, y, k)] = o;
    }
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

// The exchange of one block's six packed faces (Fig. 1(b)): face f of block
// b, packed at send_off[b][f] of the halo buffer, is copied to the receive
// segment of the neighbour's opposite face, recv_off[n][f ^ 1]. One thread
// per cell of the block's largest face, visiting the six faces in turn.
template <typename T>
__global__ void k_exchange6(const BlockDesc* desc, int b, T* halo, const int64_t* send_off, const int64_t* recv_off)
{
    const BlockDesc& d = desc[b];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
        const int n = d.nbr[f];
        if (n < 0 || q >= face_size(d, f)) continue;
        halo[recv_off[(int64_t)n * 6 + opposite_face(f)] + q] = halo[send_off[(int64_t)b * 6 + f] + q];
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
// Input check of a dense write: the lowest index whose value is not finite
// or exceeds lim in magnitude (first_bad starts at all ones).
template <typename TS>
__global__ void k_validate(const TS* src, int64_t n, double lim, unsigned long long* first_bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)src[i];
        if (!(isfinite(v) && fabs(v) <= lim)) atomicMin(first_bad, (unsigned long long)i);
    }
}

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

int tile_rows(int tw, bool f32) { return f32 ? 2 * kNT<float> / tw : 2 * kNT<double> / tw; }
int engine_threads(bool f32) { return f32 ? kNT<float> : kNT<double>; }
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
    // ny_tiles counts work-unit rows (1024 / TW for binary32); the stencil
    // engine's tile is kNT<T> / TW rows
    const int per = tile_rows(TW, sizeof(T) == 4) / (kNT<T> / TW);
    dim3 grid(nx_tiles, ny_tiles * per, 1);
    if constexpr (sizeof(T) == 8) {
        if (arith == 1) {
            // the exact-mean engines take a whole unit per CTA
            k_stencil_block<T, OP_EXACT, TW><<<dim3(nx_tiles, ny_tiles, 1), kNT<T>, kernel_bytes<T, OP_EXACT, TW>(), s>>>(
                (T*)a.pool, a.desc, a.frame, b, p);
            return;
        }
    }
    k_stencil_block<T, OP_SEQ, TW><<<grid, kNT<T>, kernel_bytes<T, OP_SEQ, TW>(), s>>>((T*)a.pool, a.desc, a.frame, b, p);
}

cudaError_t launch_stencil_block(const LaunchArgs& a, int dtype_f32, int arith, int b, int nx_tiles, int ny_tiles,
                                 int p, cudaStream_t s)
{
    if (dtype_f32) JAC_TW_DISPATCH(a.tile_w, (stencil_block_t<float, TW>(a, arith, b, nx_tiles, ny_tiles, p, s)))
    else JAC_TW_DISPATCH(a.tile_w, (stencil_block_t<double, TW>(a, arith, b, nx_tiles, ny_tiles, p, s)))
    return cudaGetLastError();
}

// Dynamic shared memory of the unit kernels: the largest over the tile widths
// the units use (units of one launch may use different widths). Only what
// those widths need is requested, so the rest of the SM stays L1 cache.
template <typename T, int OP, int TW>
static constexpr int unit_bytes_tw()
{
    if constexpr (sizeof(T) == 4 && OP == OP_SEQ) return f32_unit_bytes<TW>();
    else return kernel_bytes<T, OP, TW>();
}

template <typename T, int OP>
static int unit_bytes(int tw_mask)
{
    if (tw_mask == 0) tw_mask = 7;  // no units yet
    int n = 0;
    if (tw_mask & 1) n = std::max(n, unit_bytes_tw<T, OP, 16>());
    if (tw_mask & 2) n = std::max(n, unit_bytes_tw<T, OP, 32>());
    if (tw_mask & 4) n = std::max(n, unit_bytes_tw<T, OP, 64>());
    return n;
}

template <typename T, int OP>
static int unit_bytes_max()
{
    return unit_bytes<T, OP>(7);
}

template <int TW>
static constexpr int ring_res_bytes_tw()
{
    constexpr int a = f32_unit_bytes<TW>(), b = pair_engine_bytes<float, OP_RES32, TW, kRingRes>();
    constexpr int m = a > b ? a : b;
    return m > 256 * (int)sizeof(double) ? m : 256 * (int)sizeof(double);
}

static int ring_res_bytes(int tw_mask)
{
    if (tw_mask == 0) tw_mask = 7;
    int n = 0;
    if (tw_mask & 1) n = std::max(n, ring_res_bytes_tw<16>());
    if (tw_mask & 2) n = std::max(n, ring_res_bytes_tw<32>());
    if (tw_mask & 4) n = std::max(n, ring_res_bytes_tw<64>());
    return n;
}

template <int TW>
static constexpr int narrow_res_bytes_tw()
{
    constexpr int a = kernel_bytes<double, OP_EXACT, TW>(), b = pair_engine_bytes<double, OP_RES, TW, kRingRes>();
    constexpr int m = a > b ? a : b;
    return m > 256 * (int)sizeof(double) ? m : 256 * (int)sizeof(double);
}

static int narrow_res_bytes(int tw_mask)
{
    if (tw_mask == 0) tw_mask = 7;
    int n = 0;
    if (tw_mask & 1) n = std::max(n, narrow_res_bytes_tw<16>());
    if (tw_mask & 2) n = std::max(n, narrow_res_bytes_tw<32>());
    if (tw_mask & 4) n = std::max(n, narrow_res_bytes_tw<64>());
    return n;
}

cudaError_t launch_fused_residual_f64(const LaunchArgs& a, int p, double* partials, double* dev_out, cudaStream_t s)
{
    k_narrow_residual<1><<<a.nunits, kNT<double>, narrow_res_bytes(a.tw_mask), s>>>(
        (double*)a.pool, a.desc, a.frame, a.units, a.nunits, p, a.uexp, a.units_cap, partials, a.rcount, dev_out);
    return cudaGetLastError();
}

cudaError_t launch_fused_residual_f32(const LaunchArgs& a, int p, double* partials, double* dev_out, cudaStream_t s)
{
    k_ring_residual<1><<<a.nunits, kNT<float>, ring_res_bytes(a.tw_mask), s>>>(
        (float*)a.pool, a.desc, a.frame, a.units, a.nunits, p, partials, a.rcount, dev_out);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const LaunchArgs& a, int dtype_f32, int arith, int p, cudaStream_t s)
{
    if (dtype_f32)
        k_fused_ring<float><<<a.nunits, kNT<float>, unit_bytes<float, OP_SEQ>(a.tw_mask), s>>>((float*)a.pool, a.desc, a.units, p);
    else if (arith == 1)
        k_fused_step<double, OP_EXACT><<<a.nunits, kNT<double>, unit_bytes<double, OP_EXACT>(a.tw_mask), s>>>(
            (double*)a.pool, a.desc, a.frame, a.units, p, a.uexp, a.units_cap, a.fs);
    else
        k_fused_step<double, OP_SEQ><<<a.nunits, kNT<double>, unit_bytes<double, OP_SEQ>(a.tw_mask), s>>>(
            (double*)a.pool, a.desc, a.frame, a.units, p, a.uexp, a.units_cap, a.fs);
    return cudaGetLastError();
}

const void* persistent_kernel(int dtype_f32, int arith, int small)
{
    if (dtype_f32) return (const void*)k_persistent<float, OP_SEQ, true>;
    if (arith == 1)
        return small ? (const void*)k_persistent<double, OP_EXACT, false>
                     : (const void*)k_persistent<double, OP_EXACT, false, kMinCTAsWide>;
    return (const void*)k_persistent<double, OP_SEQ, false>;
}

int persistent_block_threads(int dtype_f32) { return dtype_f32 ? kNT<float> : kNT<double>; }

int persistent_smem_bytes(int dtype_f32, int arith, int tw_mask)
{
    if (dtype_f32) return unit_bytes<float, OP_SEQ>(tw_mask);
    return arith == 1 ? unit_bytes<double, OP_EXACT>(tw_mask) : unit_bytes<double, OP_SEQ>(tw_mask);
}

template <typename K>
static cudaError_t allow_smem(K* kernel, int bytes)
{
    return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int TW>
static cudaError_t prepare_tw()
{
    cudaError_t e = cudaSuccess;
#define JAC_ALLOW(K, BYTES) \
    if (e == cudaSuccess) e = allow_smem(K, BYTES)
    JAC_ALLOW((k_stencil_block<double, OP_EXACT, TW>), (kernel_bytes<double, OP_EXACT, TW>()));
    JAC_ALLOW((k_stencil_block<double, OP_SEQ, TW>), (kernel_bytes<double, OP_SEQ, TW>()));
    JAC_ALLOW((k_stencil_block<float, OP_SEQ, TW>), (kernel_bytes<float, OP_SEQ, TW>()));
#undef JAC_ALLOW
    return e;
}

cudaError_t prepare_kernels()
{
    cudaError_t e = prepare_tw<16>();
    if (e == cudaSuccess) e = prepare_tw<32>();
    if (e == cudaSuccess) e = prepare_tw<64>();
#define JAC_ALLOW(K, BYTES) \
    if (e == cudaSuccess) e = allow_smem(K, BYTES)
    JAC_ALLOW((k_fused_step<double, OP_EXACT>), (unit_bytes_max<double, OP_EXACT>()));
    JAC_ALLOW((k_persistent<double, OP_EXACT, false, kMinCTAsWide>), (unit_bytes_max<double, OP_EXACT>()));
    JAC_ALLOW((k_fused_step<double, OP_SEQ>), (unit_bytes_max<double, OP_SEQ>()));
    JAC_ALLOW((k_fused_ring<float>), (unit_bytes_max<float, OP_SEQ>()));
    JAC_ALLOW((k_persistent<double, OP_EXACT, false>), (unit_bytes_max<double, OP_EXACT>()));
    JAC_ALLOW((k_persistent<double, OP_SEQ, false>), (unit_bytes_max<double, OP_SEQ>()));
    JAC_ALLOW((k_persistent<float, OP_SEQ, true>), (unit_bytes_max<float, OP_SEQ>()));
    JAC_ALLOW((k_narrow_residual<1>), (narrow_res_bytes(7)));
    JAC_ALLOW((k_narrow_residual<2>), (narrow_res_bytes(7)));
    JAC_ALLOW((k_ring_residual<1>), (ring_res_bytes(7)));
    JAC_ALLOW((k_ring_residual<2>), (ring_res_bytes(7)));
#undef JAC_ALLOW
    return e;
}

cudaError_t launch_persistent(const LaunchArgs& a, const PersistentArgs& q, int dtype_f32, int arith, int ctas,
                              cudaStream_t s)
{
    if (dtype_f32)
        k_persistent<float, OP_SEQ, true><<<ctas, kNT<float>, unit_bytes<float, OP_SEQ>(a.tw_mask), s>>>(
            (float*)a.pool, a.desc, a.frame, a.units, a.nunits, q.p0, q.n_iters, q.done, q.work, q.status, q.wait_ns,
            q.hold_block, q.hold_after, a.uexp, a.units_cap, a.fs);
    else if (arith == 1)
        if (a.small)
            k_persistent<double, OP_EXACT, false><<<ctas, kNT<double>, unit_bytes<double, OP_EXACT>(a.tw_mask), s>>>(
                (double*)a.pool, a.desc, a.frame, a.units, a.nunits, q.p0, q.n_iters, q.done, q.work, q.status,
                q.wait_ns, q.hold_block, q.hold_after, a.uexp, a.units_cap, a.fs);
        else
            k_persistent<double, OP_EXACT, false, kMinCTAsWide>
                <<<ctas, kNT<double>, unit_bytes<double, OP_EXACT>(a.tw_mask), s>>>(
                    (double*)a.pool, a.desc, a.frame, a.units, a.nunits, q.p0, q.n_iters, q.done, q.work, q.status,
                    q.wait_ns, q.hold_block, q.hold_after, a.uexp, a.units_cap, a.fs);
    else
        k_persistent<double, OP_SEQ, false><<<ctas, kNT<double>, unit_bytes<double, OP_SEQ>(a.tw_mask), s>>>(
            (double*)a.pool, a.desc, a.frame, a.units, a.nunits, q.p0, q.n_iters, q.done, q.work, q.status, q.wait_ns,
            q.hold_block, q.hold_after, a.uexp, a.units_cap, a.fs);
    return cudaGetLastError();
}

cudaError_t launch_residual_partials(const LaunchArgs& a, int dtype_f32, int p, double* partials, cudaStream_t s)
{
    if (dtype_f32)
        k_ring_residual<2><<<a.nunits, kNT<float>, ring_res_bytes(a.tw_mask), s>>>(
            (float*)a.pool, a.desc, a.frame, a.units, a.nunits, p, partials, a.rcount, nullptr);
    else
        k_narrow_residual<2><<<a.nunits, kNT<double>, narrow_res_bytes(a.tw_mask), s>>>(
            (double*)a.pool, a.desc, a.frame, a.units, a.nunits, p, a.uexp, a.units_cap, partials, a.rcount, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_residual(const LaunchArgs& a, int dtype_f32, int p, double* partials, double* out,
                            cudaStream_t s)
{
    // one launch: the last unit sums the partials
    if (dtype_f32)
        k_ring_residual<2><<<a.nunits, kNT<float>, ring_res_bytes(a.tw_mask), s>>>(
            (float*)a.pool, a.desc, a.frame, a.units, a.nunits, p, partials, a.rcount, out);
    else
        k_narrow_residual<2><<<a.nunits, kNT<double>, narrow_res_bytes(a.tw_mask), s>>>(
            (double*)a.pool, a.desc, a.frame, a.units, a.nunits, p, a.uexp, a.units_cap, partials, a.rcount, out);
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

cudaError_t launch_update_region(const LaunchArgs& a, int dtype_f32, int arith, int b, int bx, int by, int p,
                                 int exterior, cudaStream_t s)
{
    const dim3 th(32, 8, 1), g((bx + 31) / 32, (by + 7) / 8, 1);
    if (dtype_f32) k_update_region<float, OP_SEQ><<<g, th, 0, s>>>((float*)a.pool, a.desc, b, p, exterior);
    else if (arith == 1) k_update_region<double, OP_EXACT><<<g, th, 0, s>>>((double*)a.pool, a.desc, b, p, exterior);
    else k_update_region<double, OP_SEQ><<<g, th, 0, s>>>((double*)a.pool, a.desc, b, p, exterior);
    return cudaGetLastError();
}

cudaError_t launch_exchange6(const LaunchArgs& a, int dtype_f32, int b, void* halo, const int64_t* send_off,
                             const int64_t* recv_off, int maxface, cudaStream_t s)
{
    const int th = 128, g = (maxface + th - 1) / th;
    if (dtype_f32) k_exchange6<float><<<g, th, 0, s>>>(a.desc, b, (float*)halo, send_off, recv_off);
    else k_exchange6<double><<<g, th, 0, s>>>(a.desc, b, (double*)halo, send_off, recv_off);
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

cudaError_t launch_validate(const void* src, int src_f32, int64_t n, double lim, unsigned long long* first_bad,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)std::min<int64_t>(want, 152 * 16);
    if (src_f32) k_validate<float><<<grid, 256, 0, s>>>((const float*)src, n, lim, first_bad);
    else k_validate<double><<<grid, 256, 0, s>>>((const double*)src, n, lim, first_bad);
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
