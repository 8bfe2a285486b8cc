// Host-side launchers of the kernels in kernels.cu, used by the runtime in
// runtime.cu. Internal; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "jac_common.cuh"

namespace jac {

struct LaunchArgs {
    void* pool;              // block storage (both buffers)
    const BlockDesc* desc;   // device block table
    const TileUnit* units;   // device tile table
    int32_t* frame;          // per instance: largest exponent field (grid frame)
    uint32_t* uexp;          // [2][units_cap]: per buffer parity and work unit, a bound on the
                             // exponent field of the unit's values there (all ones: unknown)
    int units_cap;
    const int32_t* fs;       // the units' frame-source lists (TileUnit::fs0, fsn)
    int small;               // the grid has fewer units than two waves of the exact mean's 4-CTA persistent build
    uint32_t* rcount;        // zero between launches: the last-unit counter of the binary32 residual
    int nblocks;
    int nunits;
    int tile_w;              // tile width of the update engine: 16, 32 or 64
    int tw_mask;             // tile widths present in the units: bit 0 = 16, 1 = 32, 2 = 64
};

struct PersistentArgs {
    int p0;                  // parity read by the first iteration
    int64_t n_iters;
    uint32_t* done;          // per block: tiles finished (cumulative in this launch)
    unsigned long long* work;
    DeviceStatus* status;
    int64_t wait_ns;
    int hold_block;
    int64_t hold_after;
};

// rows of a work unit's tile: 512 / tw (binary64), 1024 / tw (binary32: two columns per thread)
int tile_rows(int tw, bool f32);
int engine_threads(bool f32);
bool tile_width_supported(int tw);
int persistent_block_threads(int dtype_f32);
// small: the exact mean's three-CTA build, for grids with fewer units than two
// waves of its four-CTA one (LaunchArgs::small)
const void* persistent_kernel(int dtype_f32, int arith, int small);
// dynamic shared memory of a unit-kernel (fused, persistent) CTA whose units
// use the tile widths in tw_mask (bit 0 = 16, 1 = 32, 2 = 64): only as much
// as those widths need, so the rest of the SM's memory stays L1 cache
int persistent_smem_bytes(int dtype_f32, int arith, int tw_mask);
// raises the dynamic shared memory limit of every engine kernel on the
// current device; once per device, before the first launch or capture
cudaError_t prepare_kernels();

cudaError_t launch_stencil_block(const LaunchArgs& a, int dtype_f32, int arith, int b, int nx_tiles, int ny_tiles,
                                 int p, cudaStream_t s);
// One binary32 update iteration (k_fused_ring's result) that also writes
// rho of the grid it reads to dev_out (one launch).
cudaError_t launch_fused_residual_f32(const LaunchArgs& a, int p, double* partials, double* dev_out, cudaStream_t s);
// One binary64 iteration of the correctly rounded mean (k_fused_step's result)
// that also writes rho of the grid it reads to dev_out (one launch).
cudaError_t launch_fused_residual_f64(const LaunchArgs& a, int p, double* partials, double* dev_out, cudaStream_t s);
cudaError_t launch_fused_step(const LaunchArgs& a, int dtype_f32, int arith, int p, cudaStream_t s);
cudaError_t launch_persistent(const LaunchArgs& a, const PersistentArgs& q, int dtype_f32, int arith, int ctas,
                              cudaStream_t s);
cudaError_t launch_residual(const LaunchArgs& a, int dtype_f32, int p, double* partials, double* out,
                            cudaStream_t s);
cudaError_t launch_residual_segments(const LaunchArgs& a, int dtype_f32, int p, double* partials, const int32_t* seg,
                                     const int32_t* slot, int nseg, double* out, cudaStream_t s);
cudaError_t launch_pack_face(const LaunchArgs& a, int dtype_f32, int b, int f, int p, void* send, int n,
                             cudaStream_t s);
cudaError_t launch_unpack_face(const LaunchArgs& a, int dtype_f32, int b, int f, int p, const void* recv, int n,
                               cudaStream_t s);
cudaError_t launch_pack6(const LaunchArgs& a, int dtype_f32, int b, int p, void* send, const int64_t* faceoff,
                         int maxface, cudaStream_t s);
cudaError_t launch_unpack6(const LaunchArgs& a, int dtype_f32, int b, int p, const void* recv, const int64_t* faceoff,
                           int maxface, cudaStream_t s);
// the interior (exterior == 0: cells 1 .. b-2 on every axis) or the
// exterior (the outermost layer) of block b's update, from its ghost layer
cudaError_t launch_update_region(const LaunchArgs& a, int dtype_f32, int arith, int b, int bx, int by, int p,
                                 int exterior, cudaStream_t s);
// the six-face exchange of block b: its packed faces into the neighbours'
// receive segments of the same halo buffer
cudaError_t launch_exchange6(const LaunchArgs& a, int dtype_f32, int b, void* halo, const int64_t* send_off,
                             const int64_t* recv_off, int maxface, cudaStream_t s);
cudaError_t launch_scatter(const LaunchArgs& a, int dtype_f32, int src_f32, const void* dense, int b0, int nb,
                           int64_t dense_base, int p, cudaStream_t s);
cudaError_t launch_gather(const LaunchArgs& a, int dtype_f32, int dst_f32, void* dense, int b0, int nb,
                          int64_t dense_base, int p, cudaStream_t s);
// the lowest index of src[0 .. n) that is not finite or exceeds lim in
// magnitude, min-combined into *first_bad (which the caller sets to all ones)
cudaError_t launch_validate(const void* src, int src_f32, int64_t n, double lim, unsigned long long* first_bad,
                            cudaStream_t s);
cudaError_t launch_init_ghosts(const LaunchArgs& a, int dtype_f32, cudaStream_t s);

}  // namespace jac
