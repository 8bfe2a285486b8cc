// Internal data structures shared by the kernels and the host runtime of
// libjacobi3d. Not part of the public ABI.
//
// Storage of one block (paper Section III-C: every block keeps two copies of
// its data, the previous and the current iteration; Section II-A: each block
// carries a one-cell ghost layer filled from its neighbours):
//
//   buffer p of block b is a dense (bz+2) x (by+2) x pitch array in the
//   context's pool starting at element desc.off[p]; interior cell (i, j, k),
//   with -1 <= i <= bx, -1 <= j <= by, -1 <= k <= bz (the -1 and b* layers
//   are the ghost layer), sits at
//       off[p] + (k+1)*plane + (j+1)*pitch + OX + i,
//   OX = 128 bytes / sizeof(T), so every interior row starts on a 128-byte
//   boundary; pitch = round_up(OX + bx + 1, OX) elements, plane = pitch*(by+2).
#pragma once

#include <cstdint>

namespace jac {

constexpr int kRowAlignBytes = 128;

template <typename T>
struct Layout {
    static constexpr int OX = kRowAlignBytes / (int)sizeof(T);
};

// Face order everywhere: -x, +x, -y, +y, -z, +z.
__host__ __device__ constexpr int opposite_face(int f) { return f ^ 1; }

struct BlockDesc {
    int32_t ext[3];   // interior extents bx, by, bz
    int32_t org[3];   // origin of the block in its instance's global grid
    int32_t nbr[6];   // neighbouring block per face, or -1 at the global boundary
    int32_t inst;     // instance (grid) the block belongs to
    int32_t pitch;    // row pitch, elements
    int64_t plane;    // plane stride, elements
    int64_t off[2];   // start of buffer 0 / 1 in the pool, elements
    int64_t dense;    // start of the instance's interior in dense x-fastest arrays
    int32_t gdim[3];  // the instance's global dims
    int32_t ntiles;   // work units (tiles) of this block
    int32_t u0;       // index of the block's first work unit (its units are contiguous)
    double bc[6];     // Dirichlet value per face (used where nbr[f] < 0)
    float bcf[6];     // the same rounded to binary32 (binary32 grids)
    int32_t pad;
    alignas(8) float bcf2[6][2];  // each binary32 value twice (a constant source for 8-byte pair copies)
    alignas(16) double bc2[6][2];  // each binary64 value twice (a constant source for 16-byte pair loads)
};

// One unit of fused / persistent work: a column tile of one block over the
// planes z0 .. z1-1, tw columns wide.
struct TileUnit {
    int32_t block;
    int16_t x0, y0;
    int16_t z0, z1;
    int16_t tw;   // tile width: 16, 32 or 64 columns
    int16_t pad;
    int32_t fs0;  // its frame sources (the units whose outputs its tile reads) are fs[fs0 .. fs0 + fsn)
    int32_t fsn;  // -1: no list (the bounds of every unit of its block and neighbours are taken)
};

// Error word values written by kernels (read back by the host at syncs).
constexpr int32_t kErrNone = 0;
constexpr int32_t kErrTimeout = 1;

struct DeviceStatus {
    int32_t err;          // kErr*
    int32_t abort;        // set to stop every persistent CTA
    int32_t where_block;  // block whose wait gave up
    int32_t where_iter;   // iteration of that wait
};

}  // namespace jac
