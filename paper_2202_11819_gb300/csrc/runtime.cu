// Host runtime of libjacobi3d: the C ABI declared in include/jacobi3d.h.
//
// A context owns one global grid split into blocks (paper Section IV-A: the
// grid is decomposed into cuboid blocks, more blocks than processors when
// overdecomposed), the block table that the kernels read (per block: extents,
// origin, the six neighbour ids or the global boundary, the offsets of its two
// buffers), the two-buffer block storage (Section III-C), the halo send and
// receive buffers of the unfused flow, and the per-block streams and events
// that order that flow (Section III-A: packing, transfers and unpacking on
// high-priority streams, the update on a low-priority stream, one set per
// block).
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "jacobi3d.h"
#include "frame_sources.h"
#include "jac_common.cuh"
#include "launch.h"

using namespace jac;

namespace {

thread_local std::string g_last_error;

jac_alloc_fn g_alloc = nullptr;
jac_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return fail(JAC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(JAC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// An axis of n cells in ceil(n / b) blocks whose sizes differ by at most one,
// the larger ones first.
void split_axis(int64_t n, int32_t b, std::vector<int32_t>& size, std::vector<int32_t>& org)
{
    const int64_t nb = (n + b - 1) / b;
    const int64_t base = n / nb, rem = n % nb;
    size.resize(nb);
    org.resize(nb);
    int64_t o = 0;
    for (int64_t i = 0; i < nb; ++i) {
        size[i] = (int32_t)(base + (i < rem ? 1 : 0));
        org[i] = (int32_t)o;
        o += size[i];
    }
}

}  // namespace

// One grid of a context. A context holds one or more independent grids
// (instances, addressed by slot) whose blocks share one block table, one
// pool and one launch. Each grid's block storage is one region of the pool
// that never moves while the grid is resident; the block table is rebuilt
// from the resident grids when the set changes.
struct Instance {
    bool active;
    int64_t dims[3];
    double bc[6];
    int32_t bc_frame;   // largest exponent field over the boundary values
    int64_t region;     // byte offset of its storage in the pool
    int64_t bytes;      // bytes of its storage (both buffers, all blocks)
    std::vector<BlockDesc> geom;  // its blocks; nbr[] are indices within the grid
    int64_t dense_off;  // start of this grid in dense concatenated arrays
    int32_t b0, b1;     // its blocks [b0, b1) in the current table
    int32_t u0, u1;     // its work units [u0, u1)
    int32_t nb[3];
};

// First-fit allocator of pool regions (bytes, 256-byte granules).
struct Arena {
    char* base = nullptr;
    int64_t capacity = 0;
    int64_t used = 0;
    std::map<int64_t, int64_t> free_;  // offset -> size
    void init(void* b, int64_t cap)
    {
        base = (char*)b;
        capacity = cap;
        used = 0;
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    bool alloc(int64_t bytes, int64_t* off)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const int64_t rest = it->second - bytes;
                const int64_t noff = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[noff] = rest;
                used += bytes;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct jac_ctx {
    int device = 0;
    int64_t dims[3] = {0, 0, 0};
    int32_t req_block[3] = {0, 0, 0};
    int32_t nb[3] = {0, 0, 0};
    std::vector<Instance> inst;   // by slot
    std::vector<int32_t> hframe;  // per slot: bc_frame, the frame's starting value
    int32_t max_slots = 0;
    bool is_pool = false;         // grids can be added and removed
    bool dirty = true;            // the block table must be rebuilt
    Arena own_arena;
    Arena* arena = nullptr;       // own_arena, or one shared with other pools
    int32_t* dslot = nullptr;     // per table segment: its slot
    size_t done_cap = 0;
    int tile_w = 32;              // tile width of the update engine
    int zdepth = 0;               // planes per work unit (0: the whole block)
    // per block-width class (block x extent) tile widths overriding tile_w
    std::vector<std::pair<int32_t, int32_t>> class_tw;
    int tw_mask = 2;              // tile widths present in the units (bit 0 = 16, 1 = 32, 2 = 64)
    int dtype = JAC_F64;
    int esize = 8;
    int mode = JAC_MODE_PERSISTENT;
    int arith = JAC_ARITH_EXACT;
    double bc[6] = {0, 0, 0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    jac_alloc_fn alloc = nullptr;
    jac_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    struct Alloc {
        void* p;
        size_t bytes;
    };
    std::vector<Alloc> allocs;
    int64_t device_bytes = 0;

    std::vector<BlockDesc> hdesc;
    std::vector<TileUnit> hunits;
    std::vector<int32_t> ntx, nty;  // tiles per block in x and y
    BlockDesc* ddesc = nullptr;
    TileUnit* dunits = nullptr;
    void* pool = nullptr;
    int32_t* frame = nullptr;  // per instance: largest exponent field of the grid and its boundary
    int32_t* dseg = nullptr;   // per resident grid: first work unit (+1 entry)
    double* dres_inst = nullptr;
    size_t partials_cap = 0;
    int64_t pool_elems = 0;
    int parity = 0;
    int64_t iters = 0;
    int64_t launches = 0;

    // unfused flow
    bool halo_ready = false;
    void* halo = nullptr;                 // send region then recv region
    std::vector<int64_t> send_off, recv_off;  // per block*6 + face, elements
    std::vector<int32_t> fsize;           // per block*6 + face
    std::vector<int32_t> maxface;         // per block: its largest face with a neighbour
    void* dface = nullptr;                // device: send_off then recv_off (the six-face kernels' tables)
    std::vector<cudaStream_t> comm, comp;
    // Two event sets: one for eager issue and one used only while capturing a
    // graph (a wait may not name an event whose last record was captured).
    struct Events {
        std::vector<cudaEvent_t> sent, unpacked, updated, interior;
        cudaEvent_t fork = nullptr;
    } ev[2];
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t fgraph[2] = {nullptr, nullptr};

    // persistent
    uint32_t* done = nullptr;
    unsigned long long* work = nullptr;
    DeviceStatus* status = nullptr;
    unsigned long long* dbad = nullptr;  // input check of dense writes (lowest bad index)
    int pctas = 0;
    int64_t wait_ns = 2000000000LL;
    int hold_block = -1;
    int64_t hold_after = 0;

    // residual and I/O staging
    double* partials = nullptr;
    uint32_t* uexp = nullptr;  // [2][partials_cap] unit exponent bounds (see LaunchArgs)
    int32_t* fs = nullptr;  // the units' frame-source lists (TileUnit::fs0, fsn)
    int small = 0;          // see LaunchArgs::small
    size_t fs_cap = 0;
    double* dres = nullptr;
    uint32_t* rcount = nullptr;  // the binary32 residual's last-unit counter (zero between launches)
    void* dense = nullptr;
    size_t dense_bytes = 0;

    LaunchArgs args() const
    {
        LaunchArgs a;
        a.pool = pool;
        a.desc = ddesc;
        a.units = dunits;
        a.frame = frame;
        a.uexp = uexp;
        a.units_cap = (int)partials_cap;
        a.fs = fs;
        a.small = small;
        a.rcount = rcount;
        a.nblocks = (int)hdesc.size();
        a.nunits = (int)hunits.size();
        a.tile_w = tile_w;
        a.tw_mask = tw_mask;
        return a;
    }
    int64_t ncells() const
    {
        int64_t n = 0;
        for (const Instance& I : inst)
            if (I.active) n += I.dims[0] * I.dims[1] * I.dims[2];
        return n;
    }
    int first_active() const
    {
        for (size_t i = 0; i < inst.size(); ++i)
            if (inst[i].active) return (int)i;
        return -1;
    }
    int last_active() const
    {
        for (int i = (int)inst.size() - 1; i >= 0; --i)
            if (inst[i].active) return i;
        return -1;
    }
    int n_active() const
    {
        int n = 0;
        for (const Instance& I : inst) n += I.active ? 1 : 0;
        return n;
    }
    int64_t icells(int i) const { return inst[i].dims[0] * inst[i].dims[1] * inst[i].dims[2]; }
};

namespace {

int dev_alloc(jac_ctx* h, size_t bytes, void** out)
{
    *out = nullptr;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (h->alloc) {
        p = h->alloc(bytes, (void*)h->stream, h->alloc_user);
        if (!p) return fail(JAC_ENOMEM, "allocator hook returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    }
    h->allocs.push_back({p, bytes});
    h->device_bytes += (int64_t)bytes;
    *out = p;
    return JAC_OK;
}

void dev_free_all(jac_ctx* h)
{
    for (auto& a : h->allocs) {
        if (h->free_fn) h->free_fn(a.p, a.bytes, (void*)h->stream, h->alloc_user);
        else cudaFreeAsync(a.p, h->stream);
    }
    h->allocs.clear();
    h->device_bytes = 0;
}

int check_ctx(jac_ctx* h)
{
    if (!h) return fail(JAC_EINVAL, "null context");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return JAC_OK;
}

bool value_ok(double v, int dtype)
{
    if (!std::isfinite(v)) return false;
    const double lim = dtype == JAC_F32 ? 3.0e38 : 1.0e300;
    return std::fabs(v) <= lim;
}

void exponent_field_max(const double* bc, int dtype, int32_t& e)
{
    e = 0;
    for (int f = 0; f < 6; ++f) {
        const double v = dtype == JAC_F32 ? (double)(float)bc[f] : bc[f];
        uint64_t bits;
        memcpy(&bits, &v, 8);
        e = std::max(e, (int32_t)((bits >> 52) & 0x7FF));
    }
}

// Work units for the current tile width and z depth: per block, its column
// tiles times its z chunks, blocks in table order, so each grid's units are
// contiguous. Uploads the tile table, the per-block unit counts and the
// per-grid unit ranges.
// The tile width for blocks of x extent bx: the class override, else the
// context's width.
int class_tile_width(const jac_ctx* h, int32_t bx)
{
    for (const auto& c : h->class_tw)
        if (c.first == bx) return c.second;
    return h->tile_w;
}

// Mark every unit's exponent bound unknown (all ones), so the next
// iteration of the exact mean takes the grid's frame: after anything that
// changes the grids other than the kernels that maintain the bounds.
int forget_unit_frames(jac_ctx* h)
{
    if (h->uexp && h->partials_cap)
        CU(cudaMemsetAsync(h->uexp, 0xFF, 2 * h->partials_cap * sizeof(uint32_t), h->stream), "forget unit frames");
    return JAC_OK;
}

// The units' frame sources (frame_sources.h).
int build_frame_sources(jac_ctx* h, std::vector<int32_t>& src)
{
    const bool f32 = h->dtype == JAC_F32;
    jac::build_frame_sources(h->hunits, h->hdesc, [f32](int tw) { return tile_rows(tw, f32); }, src);
    return JAC_OK;
}

int build_units(jac_ctx* h)
{
    const int64_t nblocks = (int64_t)h->hdesc.size();
    h->tw_mask = 0;
    h->pctas = 0;  // the persistent grid depends on the widths' shared memory
    h->ntx.resize(nblocks);
    h->nty.resize(nblocks);
    h->hunits.clear();
    std::vector<int32_t> seg, slot;
    for (size_t ii = 0; ii < h->inst.size(); ++ii) {
        Instance& I = h->inst[ii];
        if (!I.active) continue;
        I.u0 = (int32_t)h->hunits.size();
        seg.push_back(I.u0);
        slot.push_back((int32_t)ii);
        for (int32_t b = I.b0; b < I.b1; ++b) {
            BlockDesc& d = h->hdesc[b];
            const int TW = class_tile_width(h, d.ext[0]), TH = tile_rows(TW, h->dtype == JAC_F32);
            h->ntx[b] = (d.ext[0] + TW - 1) / TW;
            h->nty[b] = (d.ext[1] + TH - 1) / TH;
            const int zd = h->zdepth > 0 ? h->zdepth : d.ext[2];
            const int nzc = (d.ext[2] + zd - 1) / zd;
            d.ntiles = h->ntx[b] * h->nty[b] * nzc;
            for (int zc = 0; zc < nzc; ++zc)
                for (int32_t ty = 0; ty < h->nty[b]; ++ty)
                    for (int32_t tx = 0; tx < h->ntx[b]; ++tx) {
                        TileUnit u;
                        u.block = b;
                        u.x0 = (int16_t)(tx * TW);
                        u.y0 = (int16_t)(ty * TH);
                        u.z0 = (int16_t)(zc * zd);
                        u.z1 = (int16_t)std::min(d.ext[2], (zc + 1) * zd);
                        u.tw = (int16_t)TW;
                        u.pad = 0;
                        u.fs0 = 0;
                        u.fsn = -1;  // set by build_frame_sources
                        h->tw_mask |= TW == 16 ? 1 : (TW == 32 ? 2 : 4);
                        h->hunits.push_back(u);
                    }
        }
        I.u1 = (int32_t)h->hunits.size();
    }
    // A grid with fewer units than two waves of the exact mean's four-CTA
    // persistent build takes the three-CTA one (LaunchArgs::small).
    if (!h->hunits.empty()) {
        int per_sm4 = 0, sms4 = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm4, persistent_kernel(h->dtype == JAC_F32, h->arith, 0),
                                                         persistent_block_threads(h->dtype == JAC_F32),
                                                         persistent_smem_bytes(h->dtype == JAC_F32, h->arith,
                                                                               h->tw_mask)),
           "occupancy");
        CU(cudaDeviceGetAttribute(&sms4, cudaDevAttrMultiProcessorCount, h->device), "SM count");
        h->small = (int64_t)h->hunits.size() < 2 * (int64_t)per_sm4 * sms4 ? 1 : 0;
    }
    // The last wave: when the units leave it at most half full, split its
    // units in z (each in place, so every instance's units stay together),
    // so the wave holds twice as many units of half the work.
    if (!h->hunits.empty() && !h->inst.empty()) {
        const int f32 = h->dtype == JAC_F32;
        int per_sm = 0, sms = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(f32, h->arith, h->small),
                                                         persistent_block_threads(f32),
                                                         persistent_smem_bytes(f32, h->arith, h->tw_mask)),
           "occupancy");
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "SM count");
        const int64_t slots = (int64_t)per_sm * sms, n = (int64_t)h->hunits.size();
        const int64_t r = slots > 0 ? n % slots : 0;
        if (r > 0 && 2 * r <= slots) {
            std::vector<TileUnit> tail(h->hunits.end() - r, h->hunits.end());
            h->hunits.resize(n - r);
            for (const TileUnit& u : tail) {
                if (u.z1 - u.z0 < 2) {
                    h->hunits.push_back(u);
                    continue;
                }
                TileUnit lo = u, hi = u;
                lo.z1 = hi.z0 = (int16_t)((u.z0 + u.z1) / 2);
                h->hunits.push_back(lo);
                h->hunits.push_back(hi);
            }
            // instance unit ranges and the per-block unit counts follow the new list
            seg.clear();
            for (Instance& I : h->inst) {
                if (!I.active) continue;
                I.u0 = -1;
            }
            for (int32_t b = 0; b < (int32_t)nblocks; ++b) h->hdesc[b].ntiles = 0;
            for (size_t i = 0; i < h->hunits.size(); ++i) {
                const int32_t b = h->hunits[i].block;
                h->hdesc[b].ntiles += 1;
                Instance& I = h->inst[h->hdesc[b].inst];
                if (I.u0 < 0) {
                    I.u0 = (int32_t)i;
                    seg.push_back((int32_t)i);
                }
                I.u1 = (int32_t)i + 1;
            }
        }
    }
    seg.push_back((int32_t)h->hunits.size());
    // each block's first unit (units of a block are contiguous)
    for (int32_t b = 0; b < (int32_t)nblocks; ++b) h->hdesc[b].u0 = -1;
    for (size_t i = 0; i < h->hunits.size(); ++i) {
        BlockDesc& d = h->hdesc[h->hunits[i].block];
        if (d.u0 < 0) d.u0 = (int32_t)i;
    }
    int rc;
    const size_t need = std::max<size_t>(1, h->hunits.size());
    if (need > h->partials_cap) {
        // earlier, smaller tables stay allocated until the context is destroyed
        if ((rc = dev_alloc(h, need * sizeof(TileUnit), (void**)&h->dunits))) return rc;
        if ((rc = dev_alloc(h, need * sizeof(double), (void**)&h->partials))) return rc;
        if ((rc = dev_alloc(h, 2 * need * sizeof(uint32_t), (void**)&h->uexp))) return rc;
        h->partials_cap = need;
    }
    std::vector<int32_t> fsl;
    if ((rc = build_frame_sources(h, fsl))) return rc;  // sets the units' fs0, fsn before they are copied
    if (fsl.size() > h->fs_cap || !h->fs) {
        const size_t cap = std::max<size_t>(1, fsl.size());
        if ((rc = dev_alloc(h, cap * sizeof(int32_t), (void**)&h->fs))) return rc;
        h->fs_cap = cap;
    }
    if (!fsl.empty())
        CU(cudaMemcpyAsync(h->fs, fsl.data(), fsl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream),
           "copy frame sources");
    if (nblocks > 0)
        CU(cudaMemcpyAsync(h->ddesc, h->hdesc.data(), nblocks * sizeof(BlockDesc), cudaMemcpyHostToDevice, h->stream),
           "copy block table");
    if (!h->hunits.empty())
        CU(cudaMemcpyAsync(h->dunits, h->hunits.data(), h->hunits.size() * sizeof(TileUnit), cudaMemcpyHostToDevice,
                           h->stream),
           "copy tile table");
    CU(cudaMemcpyAsync(h->dseg, seg.data(), seg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream),
       "copy unit ranges");
    if (!slot.empty())
        CU(cudaMemcpyAsync(h->dslot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream),
           "copy slot map");
    // the unit exponent bounds describe the old tables: unknown until the
    // next exact-mean iteration writes them
    if ((rc = forget_unit_frames(h))) return rc;
    // the host tables must stay valid until the copies above have run
    CU(cudaStreamSynchronize(h->stream), "table sync");
    h->pctas = 0;
    return JAC_OK;
}

// Blocks of one grid and the bytes of its storage; block offsets are relative
// to the grid's region (elements), neighbours are indices within the grid.
int64_t instance_geometry(const jac_ctx* h, Instance& I)
{
    const int OX = 128 / h->esize;
    std::vector<int32_t> sx, ox, sy, oy, sz, oz;
    split_axis(I.dims[0], h->req_block[0], sx, ox);
    split_axis(I.dims[1], h->req_block[1], sy, oy);
    split_axis(I.dims[2], h->req_block[2], sz, oz);
    I.nb[0] = (int32_t)sx.size();
    I.nb[1] = (int32_t)sy.size();
    I.nb[2] = (int32_t)sz.size();
    I.geom.clear();
    int64_t off = 0;
    for (int32_t bk = 0; bk < I.nb[2]; ++bk)
        for (int32_t bj = 0; bj < I.nb[1]; ++bj)
            for (int32_t bi = 0; bi < I.nb[0]; ++bi) {
                BlockDesc d;
                memset(&d, 0, sizeof d);
                d.ext[0] = sx[bi];
                d.ext[1] = sy[bj];
                d.ext[2] = sz[bk];
                d.org[0] = ox[bi];
                d.org[1] = oy[bj];
                d.org[2] = oz[bk];
                const int32_t ids[3] = {bi, bj, bk};
                for (int f = 0; f < 6; ++f) {
                    const int a = f >> 1, dir = (f & 1) ? 1 : -1;
                    int32_t q[3] = {bi, bj, bk};
                    q[a] = ids[a] + dir;
                    if (q[a] < 0 || q[a] >= I.nb[a]) d.nbr[f] = -1;
                    else d.nbr[f] = (int32_t)(q[0] + (int64_t)I.nb[0] * (q[1] + (int64_t)I.nb[1] * q[2]));
                    d.bc[f] = I.bc[f];
                    d.bcf[f] = (float)I.bc[f];
                    d.bcf2[f][0] = d.bcf2[f][1] = d.bcf[f];
                    d.bc2[f][0] = d.bc2[f][1] = d.bc[f];
                }
                d.pitch = (int32_t)round_up(OX + d.ext[0] + 1, OX);
                d.plane = (int64_t)d.pitch * (d.ext[1] + 2);
                const int64_t storage = d.plane * (d.ext[2] + 2);
                d.off[0] = off;
                d.off[1] = off + storage;
                off += 2 * storage;
                d.gdim[0] = (int32_t)I.dims[0];
                d.gdim[1] = (int32_t)I.dims[1];
                d.gdim[2] = (int32_t)I.dims[2];
                I.geom.push_back(d);
            }
    return off * h->esize;
}

// Place a grid in a free slot and a free region of the pool (zeroed).
int add_instance(jac_ctx* h, const int64_t dims[3], const double bc[6], int32_t* slot_out)
{
    Instance I;
    I.active = true;
    for (int a = 0; a < 3; ++a) I.dims[a] = dims[a];
    for (int f = 0; f < 6; ++f) I.bc[f] = bc[f];
    exponent_field_max(I.bc, h->dtype, I.bc_frame);
    I.bytes = instance_geometry(h, I);
    if (!h->arena->alloc(I.bytes, &I.region))
        return fail(JAC_EBUDGET, "grid of %lld bytes does not fit the pool (%lld of %lld bytes in use)",
                    (long long)I.bytes, (long long)h->arena->used, (long long)h->arena->capacity);
    const int64_t elem0 = I.region / h->esize;
    for (BlockDesc& d : I.geom) {
        d.off[0] += elem0;
        d.off[1] += elem0;
    }
    int32_t s = -1;
    for (size_t i = 0; i < h->inst.size(); ++i)
        if (!h->inst[i].active) {
            s = (int32_t)i;
            break;
        }
    if (s < 0) {
        if ((int32_t)h->inst.size() >= h->max_slots) {
            h->arena->release(I.region, I.bytes);
            return fail(JAC_EBUDGET, "all %d grid slots are in use", h->max_slots);
        }
        s = (int32_t)h->inst.size();
        h->inst.emplace_back();
        h->hframe.push_back(0);
    }
    h->inst[s] = std::move(I);
    h->hframe[s] = h->inst[s].bc_frame;
    CU(cudaMemsetAsync(h->arena->base + h->inst[s].region, 0, (size_t)h->inst[s].bytes, h->stream), "clear region");
    CU(cudaMemcpyAsync(h->frame + s, h->hframe.data() + s, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream),
       "init frame");
    CU(cudaStreamSynchronize(h->stream), "add sync");
    h->dirty = true;
    *slot_out = s;
    return JAC_OK;
}

int remove_instance(jac_ctx* h, int32_t s)
{
    if (s < 0 || s >= (int32_t)h->inst.size() || !h->inst[s].active) return fail(JAC_EINVAL, "slot %d not in use", s);
    CU(cudaStreamSynchronize(h->stream), "remove sync");
    h->arena->release(h->inst[s].region, h->inst[s].bytes);
    h->inst[s].active = false;
    h->inst[s].geom.clear();
    h->dirty = true;
    return JAC_OK;
}

void destroy_graphs(jac_ctx* h);

// Rebuild the block table from the resident grids (slot order).
int refresh(jac_ctx* h)
{
    if (!h->dirty) return JAC_OK;
    h->hdesc.clear();
    int64_t dense = 0;
    for (size_t ii = 0; ii < h->inst.size(); ++ii) {
        Instance& I = h->inst[ii];
        if (!I.active) continue;
        I.b0 = (int32_t)h->hdesc.size();
        I.dense_off = dense;
        for (const BlockDesc& g : I.geom) {
            BlockDesc d = g;
            for (int f = 0; f < 6; ++f)
                if (d.nbr[f] >= 0) d.nbr[f] += I.b0;
            d.inst = (int32_t)ii;
            d.dense = dense;
            h->hdesc.push_back(d);
        }
        I.b1 = (int32_t)h->hdesc.size();
        dense += I.dims[0] * I.dims[1] * I.dims[2];
    }
    const int64_t nblocks = (int64_t)h->hdesc.size();
    if (nblocks > (1 << 24)) return fail(JAC_EINVAL, "too many blocks");
    int rc;
    if ((size_t)nblocks > h->done_cap) {
        const size_t cap = std::max<size_t>(64, (size_t)nblocks * 2);
        if ((rc = dev_alloc(h, cap * sizeof(BlockDesc), (void**)&h->ddesc))) return rc;
        if ((rc = dev_alloc(h, cap * sizeof(uint32_t), (void**)&h->done))) return rc;
        h->done_cap = cap;
    }
    destroy_graphs(h);
    if ((rc = build_units(h))) return rc;
    if (nblocks > 0) {
        CU(launch_init_ghosts(h->args(), h->dtype == JAC_F32, h->stream), "init ghosts");
        h->launches += 1;
    }
    h->dirty = false;
    return JAC_OK;
}

int check_ready(jac_ctx* h)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    return refresh(h);
}

int ensure_halo(jac_ctx* h)
{
    if (h->halo_ready) return JAC_OK;
    const int64_t nblocks = (int64_t)h->hdesc.size();
    h->send_off.assign(nblocks * 6, 0);
    h->recv_off.assign(nblocks * 6, 0);
    h->fsize.assign(nblocks * 6, 0);
    int64_t total = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        for (int f = 0; f < 6; ++f) {
            const int a = f >> 1;
            const int32_t n = a == 0 ? d.ext[1] * d.ext[2] : (a == 1 ? d.ext[0] * d.ext[2] : d.ext[0] * d.ext[1]);
            h->fsize[b * 6 + f] = n;
            h->send_off[b * 6 + f] = total;
            total += round_up(n, 32);
        }
    }
    for (int64_t i = 0; i < nblocks * 6; ++i) h->recv_off[i] = h->send_off[i] + total;
    h->maxface.assign(nblocks, 0);
    for (int64_t b = 0; b < nblocks; ++b)
        for (int f = 0; f < 6; ++f)
            if (h->hdesc[b].nbr[f] >= 0) h->maxface[b] = std::max(h->maxface[b], h->fsize[b * 6 + f]);
    int rc;
    if ((rc = dev_alloc(h, (size_t)(2 * total) * h->esize, &h->halo))) return rc;
    if ((rc = dev_alloc(h, (size_t)(2 * nblocks * 6) * sizeof(int64_t), &h->dface))) return rc;
    CU(cudaMemcpyAsync(h->dface, h->send_off.data(), (size_t)(nblocks * 6) * sizeof(int64_t), cudaMemcpyHostToDevice,
                       h->stream),
       "face table");
    CU(cudaMemcpyAsync((int64_t*)h->dface + nblocks * 6, h->recv_off.data(), (size_t)(nblocks * 6) * sizeof(int64_t),
                       cudaMemcpyHostToDevice, h->stream),
       "face table");
    CU(cudaStreamSynchronize(h->stream), "face table");
    int lo = 0, hi = 0;
    CU(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priority range");
    h->comm.resize(nblocks);
    h->comp.resize(nblocks);
    for (int64_t b = 0; b < nblocks; ++b) {
        CU(cudaStreamCreateWithPriority(&h->comm[b], cudaStreamNonBlocking, hi), "create comm stream");
        CU(cudaStreamCreateWithPriority(&h->comp[b], cudaStreamNonBlocking, lo), "create compute stream");
    }
    for (auto& E : h->ev) {
        E.sent.resize(nblocks);
        E.unpacked.resize(nblocks);
        E.updated.resize(nblocks);
        E.interior.resize(nblocks);
        for (int64_t b = 0; b < nblocks; ++b) {
            CU(cudaEventCreateWithFlags(&E.sent[b], cudaEventDisableTiming), "create event");
            CU(cudaEventCreateWithFlags(&E.unpacked[b], cudaEventDisableTiming), "create event");
            CU(cudaEventCreateWithFlags(&E.updated[b], cudaEventDisableTiming), "create event");
            CU(cudaEventCreateWithFlags(&E.interior[b], cudaEventDisableTiming), "create event");
        }
        CU(cudaEventCreateWithFlags(&E.fork, cudaEventDisableTiming), "create event");
    }
    h->halo_ready = true;
    return JAC_OK;
}

// One iteration of the unfused flow reading buffer p (paper Fig. 1 without
// the interior/exterior split, Fig. 3): per block pack the faces that have a
// neighbour, copy them into the neighbours' receive buffers, then once all
// six halos of a block have arrived unpack them and update the block.
// `capture`: the iteration is being recorded into a graph, where the
// cross-iteration waits are implied by the order of graph launches. The
// graph holds the six-face form of pack and unpack (one kernel per block
// each, one thread per cell of the block's largest face visiting the six
// faces: Section III-D1), about half the nodes of the per-face form, which
// the eager flow keeps.
int issue_unfused(jac_ctx* h, int p, bool capture)
{
    const bool six = capture;
    const int64_t* dsend = (const int64_t*)h->dface;
    const int64_t* drecv = dsend + (int64_t)h->hdesc.size() * 6;
    const LaunchArgs a = h->args();
    const int f32 = h->dtype == JAC_F32;
    const int64_t nblocks = (int64_t)h->hdesc.size();
    char* send = (char*)h->halo;
    const size_t es = (size_t)h->esize;
    auto& E = h->ev[capture ? 1 : 0];
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        cudaStream_t s = h->comm[b];
        if (!capture) CU(cudaStreamWaitEvent(s, E.updated[b], 0), "wait updated");
        if (six) {
            if (h->maxface[b] > 0) {
                CU(launch_pack6(a, f32, (int)b, p, send, dsend + b * 6, h->maxface[b], s), "pack6");
                h->launches += 1;
            }
        } else {
            for (int f = 0; f < 6; ++f) {
                if (d.nbr[f] < 0) continue;
                CU(launch_pack_face(a, f32, (int)b, f, p, send + h->send_off[b * 6 + f] * es, h->fsize[b * 6 + f],
                                    s),
                   "pack");
                h->launches += 1;
            }
        }
        if (six) {
            // the captured form: one exchange kernel per block instead of a
            // copy node per face (a graph launch holds one iteration, so no
            // neighbour's unpack of an earlier iteration can still be reading)
            if (h->maxface[b] > 0) {
                CU(launch_exchange6(a, f32, (int)b, send, dsend, drecv, h->maxface[b], s), "exchange6");
                h->launches += 1;
            }
        } else {
            for (int f = 0; f < 6; ++f) {
                const int n = d.nbr[f];
                if (n < 0) continue;
                CU(cudaStreamWaitEvent(s, E.unpacked[n], 0), "wait unpacked");
                CU(cudaMemcpyAsync(send + h->recv_off[(int64_t)n * 6 + opposite_face(f)] * es,
                                   send + h->send_off[b * 6 + f] * es, (size_t)h->fsize[b * 6 + f] * es,
                                   cudaMemcpyDeviceToDevice, s),
                   "halo copy");
            }
        }
        CU(cudaEventRecord(E.sent[b], s), "record sent");
    }
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        cudaStream_t s = h->comm[b];
        for (int f = 0; f < 6; ++f)
            if (d.nbr[f] >= 0) CU(cudaStreamWaitEvent(s, E.sent[d.nbr[f]], 0), "wait sent");
        if (six) {
            if (h->maxface[b] > 0) {
                CU(launch_unpack6(a, f32, (int)b, p, send, drecv + b * 6, h->maxface[b], s), "unpack6");
                h->launches += 1;
            }
        } else {
            for (int f = 0; f < 6; ++f) {
                if (d.nbr[f] < 0) continue;
                CU(launch_unpack_face(a, f32, (int)b, f, p, send + h->recv_off[b * 6 + f] * es, h->fsize[b * 6 + f],
                                      s),
                   "unpack");
                h->launches += 1;
            }
        }
        CU(cudaEventRecord(E.unpacked[b], s), "record unpacked");
        CU(cudaStreamWaitEvent(h->comp[b], E.unpacked[b], 0), "wait unpacked (update)");
        CU(launch_stencil_block(a, f32, h->arith, (int)b, h->ntx[b], h->nty[b], p, h->comp[b]), "update");
        h->launches += 1;
        CU(cudaEventRecord(E.updated[b], h->comp[b]), "record updated");
    }
    return JAC_OK;
}

// One iteration of the unfused flow with the interior/exterior split (the
// manual overlap of Section II-A, Fig. 1, on the stream priorities of
// Section III-A): per block, the interior update on the low-priority compute
// stream starts as soon as the block's previous iteration is done, while the
// high-priority communication stream packs the faces, copies them to the
// neighbours and, once the neighbours' faces have arrived, unpacks them and
// updates the exterior layer. Interior and exterior write disjoint cells of
// buffer p^1; the exterior waits for the interior, whose results it reads in
// the next iteration only through the stream order, so each block's
// iteration ends with its exterior (event `updated`).
int issue_split(jac_ctx* h, int p)
{
    const LaunchArgs a = h->args();
    const int f32 = h->dtype == JAC_F32;
    const int64_t nblocks = (int64_t)h->hdesc.size();
    char* send = (char*)h->halo;
    const size_t es = (size_t)h->esize;
    auto& E = h->ev[0];
    auto inner = [&](const BlockDesc& d) { return d.ext[0] > 2 && d.ext[1] > 2 && d.ext[2] > 2; };
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        if (!inner(d)) continue;
        CU(cudaStreamWaitEvent(h->comp[b], E.updated[b], 0), "wait updated (interior)");
        CU(launch_update_region(a, f32, h->arith, (int)b, d.ext[0], d.ext[1], p, 0, h->comp[b]), "interior");
        h->launches += 1;
        CU(cudaEventRecord(E.interior[b], h->comp[b]), "record interior");
    }
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        cudaStream_t s = h->comm[b];
        CU(cudaStreamWaitEvent(s, E.updated[b], 0), "wait updated");
        for (int f = 0; f < 6; ++f) {
            if (d.nbr[f] < 0) continue;
            CU(launch_pack_face(a, f32, (int)b, f, p, send + h->send_off[b * 6 + f] * es, h->fsize[b * 6 + f], s),
               "pack");
            h->launches += 1;
        }
        for (int f = 0; f < 6; ++f) {
            const int n = d.nbr[f];
            if (n < 0) continue;
            CU(cudaStreamWaitEvent(s, E.unpacked[n], 0), "wait unpacked");
            CU(cudaMemcpyAsync(send + h->recv_off[(int64_t)n * 6 + opposite_face(f)] * es,
                               send + h->send_off[b * 6 + f] * es, (size_t)h->fsize[b * 6 + f] * es,
                               cudaMemcpyDeviceToDevice, s),
               "halo copy");
        }
        CU(cudaEventRecord(E.sent[b], s), "record sent");
    }
    for (int64_t b = 0; b < nblocks; ++b) {
        const BlockDesc& d = h->hdesc[b];
        cudaStream_t s = h->comm[b];
        for (int f = 0; f < 6; ++f)
            if (d.nbr[f] >= 0) CU(cudaStreamWaitEvent(s, E.sent[d.nbr[f]], 0), "wait sent");
        for (int f = 0; f < 6; ++f) {
            if (d.nbr[f] < 0) continue;
            CU(launch_unpack_face(a, f32, (int)b, f, p, send + h->recv_off[b * 6 + f] * es, h->fsize[b * 6 + f], s),
               "unpack");
            h->launches += 1;
        }
        CU(cudaEventRecord(E.unpacked[b], s), "record unpacked");
        if (inner(d)) CU(cudaStreamWaitEvent(s, E.interior[b], 0), "wait interior");
        CU(launch_update_region(a, f32, h->arith, (int)b, d.ext[0], d.ext[1], p, 1, s), "exterior");
        h->launches += 1;
        CU(cudaEventRecord(E.updated[b], s), "record updated");
    }
    return JAC_OK;
}

int fork_blocks(jac_ctx* h, bool capture)
{
    auto& E = h->ev[capture ? 1 : 0];
    CU(cudaEventRecord(E.fork, h->stream), "record fork");
    for (size_t b = 0; b < h->hdesc.size(); ++b) {
        CU(cudaStreamWaitEvent(h->comm[b], E.fork, 0), "fork comm");
        CU(cudaStreamWaitEvent(h->comp[b], E.fork, 0), "fork comp");
    }
    return JAC_OK;
}

// The main stream waits for every block's last update, which follows all of
// that block's packs, copies and unpacks of the iteration.
int join_blocks(jac_ctx* h, bool capture)
{
    auto& E = h->ev[capture ? 1 : 0];
    for (size_t b = 0; b < h->hdesc.size(); ++b) CU(cudaStreamWaitEvent(h->stream, E.updated[b], 0), "join");
    return JAC_OK;
}

int ensure_graph(jac_ctx* h, int p)
{
    if (h->graph[p]) return JAC_OK;
    int rc = ensure_halo(h);
    if (rc) return rc;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    const int64_t before = h->launches;
    rc = fork_blocks(h, true);
    if (!rc) rc = issue_unfused(h, p, true);
    if (!rc) rc = join_blocks(h, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->launches = before;  // recorded, not launched
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&h->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
    return JAC_OK;
}

// kernels per graph launch of the unfused flow (its six-face form: pack6,
// exchange6 and unpack6 for a block with a neighbour, then the update)
int64_t unfused_kernels(const jac_ctx* h)
{
    int64_t n = 0;
    for (size_t b = 0; b < h->hdesc.size(); ++b) n += 1 + (h->maxface[b] > 0 ? 3 : 0);
    return n;
}

constexpr int kFusedGraphIters = 2;

int ensure_fused_graph(jac_ctx* h, int p)
{
    if (h->fgraph[p]) return JAC_OK;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < kFusedGraphIters && le == cudaSuccess; ++i)
        le = launch_fused_step(h->args(), h->dtype == JAC_F32, h->arith, (p + i) & 1, h->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "capture fused step");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&h->fgraph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
    return JAC_OK;
}

void destroy_graphs(jac_ctx* h)
{
    for (int p = 0; p < 2; ++p) {
        if (h->graph[p]) cudaGraphExecDestroy(h->graph[p]);
        if (h->fgraph[p]) cudaGraphExecDestroy(h->fgraph[p]);
        h->graph[p] = h->fgraph[p] = nullptr;
    }
}

int ensure_dense(jac_ctx* h, size_t bytes)
{
    if (h->dense && h->dense_bytes >= bytes) return JAC_OK;
    // the old staging buffer is released with the context
    int rc = dev_alloc(h, bytes, &h->dense);
    if (rc) return rc;
    h->dense_bytes = bytes;
    return JAC_OK;
}

int read_status(jac_ctx* h)
{
    DeviceStatus st;
    CU(cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream), "read status");
    CU(cudaStreamSynchronize(h->stream), "sync");
    if (st.err != kErrNone) {
        CU(cudaMemsetAsync(h->status, 0, sizeof(DeviceStatus), h->stream), "clear status");
        CU(cudaStreamSynchronize(h->stream), "sync");
        return fail(JAC_ETIMEOUT, "device wait gave up (block %d, iteration %d of the launch)", st.where_block,
                    st.where_iter);
    }
    return JAC_OK;
}

// Scatter a dense x-fastest array into the blocks of instances [i0, i1)
// (their dense data back to back), resetting their frames first.
int write_dense(jac_ctx* h, int i0, int i1, const void* src, size_t n, int src_f32, bool src_on_device)
{
    if (i0 < 0 || i1 <= i0) return fail(JAC_ESTATE, "no resident grid");
    const size_t bytes = n * (src_f32 ? 4 : 8);
    const void* dsrc = src;
    if (!src_on_device) {
        int rc = ensure_dense(h, bytes);
        if (rc) return rc;
        CU(cudaMemcpyAsync(h->dense, src, bytes, cudaMemcpyHostToDevice, h->stream), "copy in");
        dsrc = h->dense;
    }
    // reject non-finite or out-of-range values before anything is overwritten
    // (binary64 values must stay within 1e300, binary32 grids' within 3e38,
    // so no sum of seven can overflow)
    {
        const double lim = src_f32 ? HUGE_VAL : (h->dtype == JAC_F32 ? 3.0e38 : 1.0e300);
        unsigned long long bad = ~0ull;
        CU(cudaMemsetAsync(h->dbad, 0xFF, sizeof(unsigned long long), h->stream), "clear check");
        CU(launch_validate(dsrc, src_f32, (int64_t)n, lim, h->dbad, h->stream), "check values");
        h->launches += 1;
        CU(cudaMemcpyAsync(&bad, h->dbad, sizeof bad, cudaMemcpyDeviceToHost, h->stream), "check result");
        CU(cudaStreamSynchronize(h->stream), "check sync");
        if (bad != ~0ull) return fail(JAC_EINVAL, "value at %llu not finite or out of range", bad);
    }
    // the scatter raises each frame to the largest exponent of the new interior
    CU(cudaMemcpyAsync(h->frame + i0, h->hframe.data() + i0, (size_t)(i1 - i0) * sizeof(int32_t),
                       cudaMemcpyHostToDevice, h->stream),
       "reset frame");
    const int b0 = h->inst[i0].b0, b1 = h->inst[i1 - 1].b1;
    CU(launch_scatter(h->args(), h->dtype == JAC_F32, src_f32, dsrc, b0, b1 - b0, h->inst[i0].dense_off, h->parity,
                      h->stream),
       "scatter");
    h->launches += 1;
    {
        const int rcf = forget_unit_frames(h);
        if (rcf) return rcf;
    }
    if (i0 == h->first_active() && i1 == h->last_active() + 1) h->iters = 0;
    if (!src_on_device) CU(cudaStreamSynchronize(h->stream), "write sync");
    return JAC_OK;
}

int read_dense(jac_ctx* h, int i0, int i1, void* dst, size_t n, int dst_f32, bool dst_on_device)
{
    if (i0 < 0 || i1 <= i0) return fail(JAC_ESTATE, "no resident grid");
    const size_t bytes = n * (dst_f32 ? 4 : 8);
    void* ddst = dst;
    if (!dst_on_device) {
        int rc = ensure_dense(h, bytes);
        if (rc) return rc;
        ddst = h->dense;
    }
    const int b0 = h->inst[i0].b0, b1 = h->inst[i1 - 1].b1;
    CU(launch_gather(h->args(), h->dtype == JAC_F32, dst_f32, ddst, b0, b1 - b0, h->inst[i0].dense_off, h->parity,
                     h->stream),
       "gather");
    h->launches += 1;
    if (!dst_on_device) {
        CU(cudaMemcpyAsync(dst, h->dense, bytes, cudaMemcpyDeviceToHost, h->stream), "copy out");
        return read_status(h);
    }
    return JAC_OK;
}

int sync_stream(jac_ctx* h)
{
    CU(cudaStreamSynchronize(h->stream), "sync");
    return JAC_OK;
}

// Stream, allocator and the fixed-size device tables (per slot and status).
// Per-device one-time kernel setup (dynamic shared-memory limits).
static cudaError_t prepare_device(int dev)
{
    static std::mutex mu;
    static std::vector<char> done;
    std::lock_guard<std::mutex> lock(mu);
    if ((size_t)dev < done.size() && done[dev]) return cudaSuccess;
    const cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    if ((size_t)dev >= done.size()) done.resize(dev + 1, 0);
    done[dev] = 1;
    return cudaSuccess;
}

int open_ctx(jac_ctx* h, void* stream)
{
    h->alloc = g_alloc;
    h->free_fn = g_free;
    h->alloc_user = g_alloc_user;
    cudaError_t e;
    if (stream) {
        h->stream = (cudaStream_t)stream;
        e = cudaStreamGetDevice(h->stream, &h->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetDevice");
        cudaSetDevice(h->device);
    } else {
        cudaGetDevice(&h->device);
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        h->own_stream = true;
    }
    if ((e = prepare_device(h->device)) != cudaSuccess) return cuda_fail(e, "kernel shared-memory limits");
    const size_t ns = (size_t)std::max(1, h->max_slots);
    int rc;
    if ((rc = dev_alloc(h, sizeof(unsigned long long), (void**)&h->work))) return rc;
    if ((rc = dev_alloc(h, sizeof(DeviceStatus), (void**)&h->status))) return rc;
    if ((rc = dev_alloc(h, sizeof(unsigned long long), (void**)&h->dbad))) return rc;
    if ((rc = dev_alloc(h, sizeof(double), (void**)&h->dres))) return rc;
    if ((rc = dev_alloc(h, sizeof(uint32_t), (void**)&h->rcount))) return rc;
    if ((rc = dev_alloc(h, ns * sizeof(double), (void**)&h->dres_inst))) return rc;
    if ((rc = dev_alloc(h, ns * sizeof(int32_t), (void**)&h->frame))) return rc;
    if ((rc = dev_alloc(h, (ns + 1) * sizeof(int32_t), (void**)&h->dseg))) return rc;
    if ((rc = dev_alloc(h, ns * sizeof(int32_t), (void**)&h->dslot))) return rc;
    CU(cudaMemsetAsync(h->status, 0, sizeof(DeviceStatus), h->stream), "clear status");
    CU(cudaMemsetAsync(h->rcount, 0, sizeof(uint32_t), h->stream), "clear residual counter");
    return JAC_OK;
}

// A pool context whose regions come from an arena owned by someone else
// (the server shares one arena between its binary64 and binary32 pools).
int create_pool_shared(jac_ctx** out, int32_t dtype, Arena* arena, int32_t max_grids, int32_t bx, int32_t by,
                       int32_t bz, void* stream)
{
    jac_ctx* h = new jac_ctx();
    h->req_block[0] = bx;
    h->req_block[1] = by;
    h->req_block[2] = bz;
    h->dtype = dtype;
    h->esize = dtype == JAC_F32 ? 4 : 8;
    h->arith = dtype == JAC_F32 ? JAC_ARITH_SEQ : JAC_ARITH_EXACT;
    h->max_slots = max_grids;
    h->is_pool = true;
    h->arena = arena;
    h->pool = arena->base;
    int rc = open_ctx(h, stream);
    if (!rc) rc = refresh(h);
    if (!rc) rc = sync_stream(h);
    if (rc) {
        std::string msg = g_last_error;
        jac_destroy(h);
        g_last_error = msg;
        return rc;
    }
    *out = h;
    return JAC_OK;
}

int64_t range_cells(const jac_ctx* h, int i0, int i1)
{
    int64_t n = 0;
    for (int i = i0; i < i1; ++i) n += h->icells(i);
    return n;
}

int create_ctx(jac_ctx** out, int32_t n_inst, const int64_t* dims, int32_t bx, int32_t by, int32_t bz, int32_t dtype,
               const double* bc, void* stream)
{
    if (!out) return fail(JAC_EINVAL, "null output pointer");
    *out = nullptr;
    if (n_inst < 1 || !dims || !bc) return fail(JAC_EINVAL, "need n_inst >= 1, dims and boundary values");
    if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256)
        return fail(JAC_EINVAL, "block dims must be in [1, 256]");
    if (dtype != JAC_F64 && dtype != JAC_F32) return fail(JAC_EINVAL, "dtype must be JAC_F64 or JAC_F32");
    for (int32_t i = 0; i < n_inst; ++i) {
        for (int a = 0; a < 3; ++a) {
            const int64_t n = dims[3 * i + a];
            if (n < 1 || n > (1 << 30)) return fail(JAC_EINVAL, "instance %d: grid dims must be in [1, 2^30]", i);
        }
        if (n_inst == 1 && (bx > dims[0] || by > dims[1] || bz > dims[2]))
            return fail(JAC_EINVAL, "block dims must not exceed grid dims");
        for (int f = 0; f < 6; ++f)
            if (!value_ok(bc[6 * i + f], dtype))
                return fail(JAC_EINVAL, "instance %d: boundary value %d not finite or out of range", i, f);
    }
    jac_ctx* h = new jac_ctx();
    h->req_block[0] = bx;
    h->req_block[1] = by;
    h->req_block[2] = bz;
    h->dtype = dtype;
    h->esize = dtype == JAC_F32 ? 4 : 8;
    h->arith = dtype == JAC_F32 ? JAC_ARITH_SEQ : JAC_ARITH_EXACT;
    h->max_slots = n_inst;
    for (int a = 0; a < 3; ++a) h->dims[a] = n_inst == 1 ? dims[a] : 0;
    for (int f = 0; f < 6; ++f) h->bc[f] = bc[f];
    int rc = open_ctx(h, stream);
    if (rc) {
        std::string msg = g_last_error;
        jac_destroy(h);
        g_last_error = msg;
        return rc;
    }
    // one region per grid, back to back: size the pool to their sum
    int64_t total = 0;
    for (int32_t i = 0; i < n_inst; ++i) {
        Instance I;
        for (int a = 0; a < 3; ++a) I.dims[a] = dims[3 * i + a];
        for (int f = 0; f < 6; ++f) I.bc[f] = bc[6 * i + f];
        total += (instance_geometry(h, I) + 255) / 256 * 256;
    }
    void* pool = nullptr;
    if (!(rc = dev_alloc(h, (size_t)total, &pool))) {
        h->own_arena.init(pool, total);
        h->arena = &h->own_arena;
        h->pool = pool;
        for (int32_t i = 0; i < n_inst && !rc; ++i) {
            int32_t slot;
            rc = add_instance(h, dims + 3 * i, bc + 6 * i, &slot);
        }
    }
    if (!rc) rc = refresh(h);
    if (!rc) rc = sync_stream(h);
    if (rc) {
        std::string msg = g_last_error;
        jac_destroy(h);
        g_last_error = msg;
        return rc;
    }
    *out = h;
    return JAC_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

const char* jac_strerror(int code)
{
    switch (code) {
        case JAC_OK: return "ok";
        case JAC_EINVAL: return "invalid argument";
        case JAC_ENOMEM: return "out of memory";
        case JAC_ECUDA: return "CUDA error";
        case JAC_ETIMEOUT: return "device wait timed out";
        case JAC_EBUDGET: return "HBM budget exceeded";
        case JAC_ESTATE: return "invalid state";
        default: return "unknown error";
    }
}

const char* jac_last_error(void) { return g_last_error.c_str(); }

// ---- host buffers
namespace {

std::mutex g_host_mu;
struct HostBuf {
    size_t len;
    bool mapped;  // huge-page mapping (munmap) rather than cudaHostAlloc
};
std::map<void*, HostBuf> g_host;

// The transparent huge page size when the kernel offers them on request
// (mode "always" or "madvise"), else 0.
size_t thp_bytes()
{
    static const size_t hp = [] {
        size_t v = 0;
        if (FILE* f = fopen("/sys/kernel/mm/transparent_hugepage/enabled", "r")) {
            char buf[128] = {0};
            const bool on = fgets(buf, sizeof buf, f) && (strstr(buf, "[always]") || strstr(buf, "[madvise]"));
            fclose(f);
            if (on) {
                if (FILE* g = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
                    unsigned long long x = 0;
                    if (fscanf(g, "%llu", &x) == 1) v = (size_t)x;
                    fclose(g);
                }
            }
        }
        return v;
    }();
    return hp;
}

constexpr size_t kHostHugeMin = size_t(64) << 20;  // smaller requests get base pages

// Bytes of [p, p + len) the kernel backs with transparent huge pages (the
// AnonHugePages of the mappings it overlaps in /proc/self/smaps).
size_t huge_bytes(const void* p, size_t len)
{
    FILE* f = fopen("/proc/self/smaps", "r");
    if (!f) return 0;
    char line[512];
    bool in = false;
    size_t kb = 0;
    const uintptr_t a = (uintptr_t)p, e = a + len;
    while (fgets(line, sizeof line, f)) {
        unsigned long lo = 0, hi = 0;
        if (sscanf(line, "%lx-%lx", &lo, &hi) == 2) {  // a mapping's header line
            in = lo < e && hi > a;
            continue;
        }
        unsigned long v = 0;
        if (in && strncmp(line, "AnonHugePages:", 14) == 0 && sscanf(line + 14, "%lu", &v) == 1) kb += v;
    }
    fclose(f);
    return kb * 1024;
}

// Prefer the current GPU's nearest host NUMA node for the pages of [p, p +
// len), so that they are not faulted in on whichever node the calling thread
// happens to run (a far node halves or worse the device's writes to them).
// Best effort: nothing changes where the attribute or the call is missing.
void prefer_gpu_numa_node(void* p, size_t len)
{
    int dev = 0, node = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (cudaDeviceGetAttribute(&node, cudaDevAttrHostNumaId, dev) != cudaSuccess || node < 0 || node >= 63) return;
    unsigned long mask = 1ul << node;
    constexpr long kMpolPreferred = 1;
    syscall(SYS_mbind, p, len, kMpolPreferred, &mask, (unsigned long)(8 * sizeof mask), 0u);
}

}  // namespace

void* jac_host_alloc(size_t bytes)
{
    if (bytes == 0) {
        fail(JAC_EINVAL, "jac_host_alloc: zero bytes");
        return nullptr;
    }
    const size_t hp = thp_bytes();
    if (hp && bytes >= kHostHugeMin) {
        const size_t len = (bytes + hp - 1) / hp * hp;
        void* raw = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
        if (raw != MAP_FAILED) {
            // keep the huge-page-aligned part
            const uintptr_t r = (uintptr_t)raw, a = (r + hp - 1) / hp * hp;
            if (a > r) munmap(raw, a - r);
            if (r + len + hp > a + len) munmap((void*)(a + len), r + len + hp - (a + len));
            void* p = (void*)a;
            madvise(p, len, MADV_HUGEPAGE);
            prefer_gpu_numa_node(p, len);
            memset(p, 0, len);  // fault the pages in (huge, on that node) before they are pinned
            constexpr int kMadvCollapse = 25;  // synchronous collapse where the faults got base pages
            if (huge_bytes(p, len) < len) madvise(p, len, kMadvCollapse);
            // registered base pages are slower to copy than the driver's pinned memory: keep the
            // mapping only when (nearly) all of it is on huge pages
            if (huge_bytes(p, len) >= len - len / 16) {
                const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterPortable);
                if (e == cudaSuccess) {
                    std::lock_guard<std::mutex> lock(g_host_mu);
                    g_host[p] = HostBuf{len, true};
                    return p;
                }
                munmap(p, len);
                cuda_fail(e, "jac_host_alloc: cudaHostRegister");
                return nullptr;
            }
            munmap(p, len);
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cuda_fail(e, "jac_host_alloc: cudaHostAlloc");
        return nullptr;
    }
    memset(p, 0, bytes);
    std::lock_guard<std::mutex> lock(g_host_mu);
    g_host[p] = HostBuf{bytes, false};
    return p;
}

int jac_host_alloc_kind(const void* p)
{
    std::lock_guard<std::mutex> lock(g_host_mu);
    auto it = g_host.find(const_cast<void*>(p));
    if (it == g_host.end()) return -1;
    return it->second.mapped ? 1 : 0;
}

int jac_host_free(void* p)
{
    if (!p) return JAC_OK;
    HostBuf b;
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host.find(p);
        if (it == g_host.end()) return fail(JAC_EINVAL, "jac_host_free: not a pointer from jac_host_alloc");
        b = it->second;
        g_host.erase(it);
    }
    if (b.mapped) {
        const cudaError_t e = cudaHostUnregister(p);
        munmap(p, b.len);
        if (e != cudaSuccess) return cuda_fail(e, "jac_host_free: cudaHostUnregister");
        return JAC_OK;
    }
    CU(cudaFreeHost(p), "jac_host_free: cudaFreeHost");
    return JAC_OK;
}

int jac_set_allocator(jac_alloc_fn alloc, jac_free_fn free_fn, void* user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(JAC_EINVAL, "alloc and free must both be set or both NULL");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return JAC_OK;
}

int jac_create(jac_ctx** out, int64_t nx, int64_t ny, int64_t nz, int32_t bx, int32_t by, int32_t bz, int32_t dtype,
               const double bc[6], void* stream)
{
    const int64_t dims[3] = {nx, ny, nz};
    if (!bc) return fail(JAC_EINVAL, "null boundary values");
    return create_ctx(out, 1, dims, bx, by, bz, dtype, bc, stream);
}

int jac_create_batch(jac_ctx** out, int32_t n_inst, const int64_t* dims, int32_t bx, int32_t by, int32_t bz,
                     int32_t dtype, const double* bc, void* stream)
{
    return create_ctx(out, n_inst, dims, bx, by, bz, dtype, bc, stream);
}

int jac_destroy(jac_ctx* h)
{
    if (!h) return JAC_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto s : h->comm) cudaStreamSynchronize(s);
    for (auto s : h->comp) cudaStreamSynchronize(s);
    destroy_graphs(h);
    for (auto s : h->comm) cudaStreamDestroy(s);
    for (auto s : h->comp) cudaStreamDestroy(s);
    for (auto& E : h->ev) {
        for (auto e : E.sent) cudaEventDestroy(e);
        for (auto e : E.unpacked) cudaEventDestroy(e);
        for (auto e : E.updated) cudaEventDestroy(e);
        if (E.fork) cudaEventDestroy(E.fork);
    }
    dev_free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return JAC_OK;
}

int jac_set_mode(jac_ctx* h, int32_t mode)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (mode < JAC_MODE_UNFUSED || mode > JAC_MODE_SPLIT) return fail(JAC_EINVAL, "unknown mode %d", mode);
    if (h->is_pool && (mode == JAC_MODE_UNFUSED || mode == JAC_MODE_GRAPH || mode == JAC_MODE_SPLIT))
        return fail(JAC_EINVAL, "pools run the fused or persistent forms only");
    h->mode = mode;
    return JAC_OK;
}

int jac_set_arith(jac_ctx* h, int32_t arith)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (arith != JAC_ARITH_SEQ && arith != JAC_ARITH_EXACT) return fail(JAC_EINVAL, "unknown arith %d", arith);
    if (h->dtype == JAC_F32 && arith != JAC_ARITH_SEQ) return fail(JAC_EINVAL, "F32 contexts use JAC_ARITH_SEQ");
    if (arith == h->arith) return JAC_OK;
    destroy_graphs(h);
    h->arith = arith;
    // the last wave's unit split follows the persistent kernel's occupancy,
    // which depends on the rule
    return h->dirty ? JAC_OK : build_units(h);
}

int jac_write(jac_ctx* h, const double* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return write_dense(h, h->first_active(), h->last_active() + 1, host, n_cells, 0, false);
}

int jac_write_f32(jac_ctx* h, const float* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if (h->dtype != JAC_F32) return fail(JAC_EINVAL, "jac_write_f32 needs an F32 context");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return write_dense(h, h->first_active(), h->last_active() + 1, host, n_cells, 1, false);
}

int jac_write_device(jac_ctx* h, const void* dev, size_t n_cells, int32_t dtype)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!dev) return fail(JAC_EINVAL, "null device pointer");
    if (dtype != h->dtype) return fail(JAC_EINVAL, "dtype must equal the context's dtype");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return write_dense(h, h->first_active(), h->last_active() + 1, dev, n_cells, dtype == JAC_F32, true);
}

int jac_read(jac_ctx* h, double* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return read_dense(h, h->first_active(), h->last_active() + 1, host, n_cells, 0, false);
}

int jac_read_f32(jac_ctx* h, float* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if (h->dtype != JAC_F32) return fail(JAC_EINVAL, "jac_read_f32 needs an F32 context");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return read_dense(h, h->first_active(), h->last_active() + 1, host, n_cells, 1, false);
}

int jac_read_device(jac_ctx* h, void* dev, size_t n_cells, int32_t dtype)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!dev) return fail(JAC_EINVAL, "null device pointer");
    if (dtype != h->dtype && !(h->dtype == JAC_F32 && dtype == JAC_F64))
        return fail(JAC_EINVAL, "dtype must be the context's dtype (or F64 for an F32 context)");
    if ((int64_t)n_cells != h->ncells()) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->ncells());
    return read_dense(h, h->first_active(), h->last_active() + 1, dev, n_cells, dtype == JAC_F32, true);
}

int jac_iterate(jac_ctx* h, int64_t n)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (n < 0) return fail(JAC_EINVAL, "n_iters must be >= 0");
    if (n == 0 || h->hunits.empty()) return JAC_OK;
    const int f32 = h->dtype == JAC_F32;
    // only the fused and persistent forms of the exact mean keep the unit
    // exponent bounds; after any other iteration they are unknown
    const bool keeps = !f32 && h->arith == JAC_ARITH_EXACT &&
                       (h->mode == JAC_MODE_FUSED || h->mode == JAC_MODE_GRAPH_FUSED || h->mode == JAC_MODE_PERSISTENT);
    if (!keeps && (rc = forget_unit_frames(h))) return rc;
    switch (h->mode) {
        case JAC_MODE_FUSED:
            for (int64_t i = 0; i < n; ++i) {
                CU(launch_fused_step(h->args(), f32, h->arith, h->parity, h->stream), "fused step");
                h->launches += 1;
                h->parity ^= 1;
            }
            break;
        case JAC_MODE_GRAPH_FUSED: {
            int64_t i = 0;
            for (; i + kFusedGraphIters <= n; i += kFusedGraphIters) {
                if ((rc = ensure_fused_graph(h, h->parity))) return rc;
                CU(cudaGraphLaunch(h->fgraph[h->parity], h->stream), "graph launch");
                h->launches += kFusedGraphIters;
                if (kFusedGraphIters & 1) h->parity ^= 1;
            }
            for (; i < n; ++i) {
                CU(launch_fused_step(h->args(), f32, h->arith, h->parity, h->stream), "fused step");
                h->launches += 1;
                h->parity ^= 1;
            }
            break;
        }
        case JAC_MODE_UNFUSED:
            if ((rc = ensure_halo(h))) return rc;
            if ((rc = fork_blocks(h, false))) return rc;
            for (int64_t i = 0; i < n; ++i) {
                if ((rc = issue_unfused(h, h->parity, false))) return rc;
                h->parity ^= 1;
            }
            if ((rc = join_blocks(h, false))) return rc;
            break;
        case JAC_MODE_SPLIT:
            if ((rc = ensure_halo(h))) return rc;
            if ((rc = fork_blocks(h, false))) return rc;
            for (int64_t i = 0; i < n; ++i) {
                if ((rc = issue_split(h, h->parity))) return rc;
                h->parity ^= 1;
            }
            if ((rc = join_blocks(h, false))) return rc;
            break;
        case JAC_MODE_GRAPH:
            for (int64_t i = 0; i < n; ++i) {
                if ((rc = ensure_graph(h, h->parity))) return rc;
                CU(cudaGraphLaunch(h->graph[h->parity], h->stream), "graph launch");
                h->launches += unfused_kernels(h);
                h->parity ^= 1;
            }
            break;
        case JAC_MODE_PERSISTENT: {
            if (h->pctas == 0) {
                int per_sm = 0, sms = 0;
                CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(f32, h->arith, h->small),
                                                                 persistent_block_threads(f32),
                                                                 persistent_smem_bytes(f32, h->arith, h->tw_mask)),
                   "occupancy");
                CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "SM count");
                h->pctas = std::max(1, std::min(per_sm * sms, (int)h->hunits.size()));
            }
            // counters are 32-bit: at most 2^32 / max tiles per block iterations per launch
            int32_t maxt = 1;
            for (const BlockDesc& d : h->hdesc) maxt = std::max(maxt, d.ntiles);
            const int64_t chunk = std::max<int64_t>(1, (int64_t)(0xFFFFFFF0u / (uint32_t)maxt) - 1);
            for (int64_t done_it = 0; done_it < n;) {
                const int64_t m = std::min(chunk, n - done_it);
                CU(cudaMemsetAsync(h->done, 0, h->hdesc.size() * sizeof(uint32_t), h->stream), "clear counters");
                CU(cudaMemsetAsync(h->work, 0, sizeof(unsigned long long), h->stream), "clear work");
                CU(cudaMemsetAsync(&h->status->abort, 0, sizeof(int32_t), h->stream), "clear abort");
                PersistentArgs q;
                q.p0 = h->parity;
                q.n_iters = m;
                q.done = h->done;
                q.work = h->work;
                q.status = h->status;
                q.wait_ns = h->wait_ns;
                q.hold_block = h->hold_block;
                q.hold_after = h->hold_after;
                CU(launch_persistent(h->args(), q, f32, h->arith, h->pctas, h->stream), "persistent");
                h->launches += 1;
                if (m & 1) h->parity ^= 1;
                done_it += m;
            }
            break;
        }
        default:
            return fail(JAC_ESTATE, "bad mode");
    }
    h->iters += n;
    return JAC_OK;
}

int jac_residual_device(jac_ctx* h, double* dev_out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!dev_out) return fail(JAC_EINVAL, "null output pointer");
    if (h->hunits.empty()) return fail(JAC_ESTATE, "no resident grid");
    CU(launch_residual(h->args(), h->dtype == JAC_F32, h->parity, h->partials, dev_out, h->stream), "residual");
    h->launches += 1;
    return JAC_OK;
}

int jac_iterate_residual(jac_ctx* h, int64_t n, int64_t every, double* dev_out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (n < 0) return fail(JAC_EINVAL, "n_iters must be >= 0");
    if (every < 1) return fail(JAC_EINVAL, "every must be >= 1");
    if (n == 0) return JAC_OK;
    if (!dev_out) return fail(JAC_EINVAL, "null output pointer");
    if (h->hunits.empty()) return fail(JAC_ESTATE, "no resident grid");
    // the fused forms (binary32, or binary64 with the correctly rounded mean):
    // the residual of u^k comes from the launch that computes u^(k+1);
    // elsewhere the residual launch precedes the chunk
    const bool fused_form = h->mode == JAC_MODE_FUSED || h->mode == JAC_MODE_GRAPH_FUSED;
    const bool f32 = h->dtype == JAC_F32;
    const bool fuse = fused_form && (f32 || h->arith == JAC_ARITH_EXACT);
    for (int64_t i = 0, j = 0; i < n; i += every, ++j) {
        const int64_t m = std::min(every, n - i);
        if (fuse) {
            CU(f32 ? launch_fused_residual_f32(h->args(), h->parity, h->partials, dev_out + j, h->stream)
                   : launch_fused_residual_f64(h->args(), h->parity, h->partials, dev_out + j, h->stream),
               "fused residual");
            h->launches += 1;
            h->parity ^= 1;
            h->iters += 1;
            if (m > 1 && (rc = jac_iterate(h, m - 1))) return rc;
        } else {
            if ((rc = jac_residual_device(h, dev_out + j))) return rc;
            if ((rc = jac_iterate(h, m))) return rc;
        }
    }
    return JAC_OK;
}

int jac_residual(jac_ctx* h, double* out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!out) return fail(JAC_EINVAL, "null output pointer");
    if ((rc = jac_residual_device(h, h->dres))) return rc;
    CU(cudaMemcpyAsync(out, h->dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy residual");
    return read_status(h);
}

int jac_sync(jac_ctx* h)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    return read_status(h);
}

int jac_info(jac_ctx* h, jac_info_t* info)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (!info) return fail(JAC_EINVAL, "null info pointer");
    memset(info, 0, sizeof *info);
    for (int a = 0; a < 3; ++a) {
        info->dims[a] = h->dims[a];
        info->block[a] = h->req_block[a];
        info->nblocks[a] = h->nb[a];
    }
    info->dtype = h->dtype;
    info->mode = h->mode;
    info->arith = h->arith;
    info->persistent_ctas = h->pctas;
    info->iterations = h->iters;
    info->device_bytes = h->device_bytes;
    info->kernel_launches = h->launches;
    info->n_instances = h->n_active();
    info->tile_w = h->tile_w;
    info->zdepth = h->zdepth;
    info->n_units = (int32_t)h->hunits.size();
    info->n_blocks = (int32_t)h->hdesc.size();
    return JAC_OK;
}

int jac_write_instance(jac_ctx* h, int32_t i, const double* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (i < 0 || i >= (int32_t)h->inst.size() || !h->inst[i].active) return fail(JAC_EINVAL, "grid slot %d not in use", i);
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if ((int64_t)n_cells != h->icells(i)) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->icells(i));
    return write_dense(h, i, i + 1, host, n_cells, 0, false);
}

int jac_write_instance_device(jac_ctx* h, int32_t i, const void* dev, size_t n_cells, int32_t dtype)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (i < 0 || i >= (int32_t)h->inst.size() || !h->inst[i].active) return fail(JAC_EINVAL, "grid slot %d not in use", i);
    if (!dev) return fail(JAC_EINVAL, "null device pointer");
    if (dtype != h->dtype) return fail(JAC_EINVAL, "dtype must equal the context's dtype");
    if ((int64_t)n_cells != h->icells(i)) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->icells(i));
    return write_dense(h, i, i + 1, dev, n_cells, dtype == JAC_F32, true);
}

int jac_read_instance(jac_ctx* h, int32_t i, double* host, size_t n_cells)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (i < 0 || i >= (int32_t)h->inst.size() || !h->inst[i].active) return fail(JAC_EINVAL, "grid slot %d not in use", i);
    if (!host) return fail(JAC_EINVAL, "null host pointer");
    if ((int64_t)n_cells != h->icells(i)) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->icells(i));
    return read_dense(h, i, i + 1, host, n_cells, 0, false);
}

int jac_read_instance_device(jac_ctx* h, int32_t i, void* dev, size_t n_cells, int32_t dtype)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (i < 0 || i >= (int32_t)h->inst.size() || !h->inst[i].active) return fail(JAC_EINVAL, "grid slot %d not in use", i);
    if (!dev) return fail(JAC_EINVAL, "null device pointer");
    if (dtype != h->dtype && !(h->dtype == JAC_F32 && dtype == JAC_F64))
        return fail(JAC_EINVAL, "dtype must be the context's dtype (or F64 for an F32 context)");
    if ((int64_t)n_cells != h->icells(i)) return fail(JAC_EINVAL, "n_cells %zu != %lld", n_cells, (long long)h->icells(i));
    return read_dense(h, i, i + 1, dev, n_cells, dtype == JAC_F32, true);
}

int jac_residual_instances_device(jac_ctx* h, double* dev_out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!dev_out) return fail(JAC_EINVAL, "null output pointer");
    if (h->hunits.empty()) return JAC_OK;
    CU(launch_residual_segments(h->args(), h->dtype == JAC_F32, h->parity, h->partials, h->dseg, h->dslot,
                                h->n_active(), dev_out, h->stream),
       "residual");
    h->launches += 2;
    return JAC_OK;
}

int jac_residual_instances(jac_ctx* h, double* out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!out) return fail(JAC_EINVAL, "null output pointer");
    if ((rc = jac_residual_instances_device(h, h->dres_inst))) return rc;
    if (!h->inst.empty())
        CU(cudaMemcpyAsync(out, h->dres_inst, h->inst.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "copy residuals");
    rc = read_status(h);
    for (size_t i = 0; i < h->inst.size(); ++i)
        if (!h->inst[i].active) out[i] = std::nan("");
    return rc;
}

int jac_set_tile(jac_ctx* h, int32_t tile_w, int32_t zdepth)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!tile_width_supported(tile_w)) return fail(JAC_EINVAL, "tile width must be 16, 32 or 64");
    if (zdepth < 0 || zdepth > 256) return fail(JAC_EINVAL, "z depth must be in [0, 256]");
    if (tile_w == h->tile_w && zdepth == h->zdepth && h->class_tw.empty()) return JAC_OK;
    CU(cudaStreamSynchronize(h->stream), "tile sync");
    h->tile_w = tile_w;
    h->zdepth = zdepth;
    h->class_tw.clear();
    destroy_graphs(h);
    return build_units(h);
}

int jac_set_tile_class(jac_ctx* h, int32_t block_x, int32_t tile_w)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (block_x < 1) return fail(JAC_EINVAL, "block x extent must be >= 1");
    if (tile_w != 0 && !tile_width_supported(tile_w)) return fail(JAC_EINVAL, "tile width must be 0, 16, 32 or 64");
    CU(cudaStreamSynchronize(h->stream), "tile sync");
    auto it = std::find_if(h->class_tw.begin(), h->class_tw.end(),
                           [&](const std::pair<int32_t, int32_t>& c) { return c.first == block_x; });
    if (tile_w == 0) {
        if (it != h->class_tw.end()) h->class_tw.erase(it);
    } else if (it != h->class_tw.end()) {
        it->second = tile_w;
    } else {
        h->class_tw.emplace_back(block_x, tile_w);
    }
    destroy_graphs(h);
    return build_units(h);
}

// Time every (tile width, z depth) pair for the current mode on the context
// itself and keep the fastest; then, when the blocks come in several x
// extents (block-width classes), refine the width class by class (largest
// classes first), keeping a change only when the whole launch gets faster.
// The grid and iteration count are put back as they were.
int jac_autotune(jac_ctx* h, int32_t trial_iters, jac_tune_t* result)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (trial_iters < 1) return fail(JAC_EINVAL, "trial_iters must be >= 1");
    if (h->hunits.empty()) return fail(JAC_ESTATE, "no resident grid");
    int64_t extent = 0;
    for (const Instance& I : h->inst)
        if (I.active) extent = std::max(extent, I.region + I.bytes);
    const size_t bytes = (size_t)extent;
    void* snap = nullptr;
    CU(cudaMallocAsync(&snap, bytes, h->stream), "autotune snapshot");
    CU(cudaMemcpyAsync(snap, h->pool, bytes, cudaMemcpyDeviceToDevice, h->stream), "snapshot");
    const int parity0 = h->parity;
    const int64_t iters0 = h->iters;
    int32_t max_bz = 1;
    for (const BlockDesc& d : h->hdesc) max_bz = std::max(max_bz, d.ext[2]);
    const int widths[3] = {16, 32, 64};
    const int depths[4] = {0, 64, 32, 16};
    jac_tune_t best;
    memset(&best, 0, sizeof best);
    best.ms_per_iter = 1e300;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0), "event");
    CU(cudaEventCreate(&e1), "event");
    auto time_it = [&](double* per) -> int {
        int r;
        if ((r = jac_iterate(h, 1))) return r;  // builds graphs / streams outside the timing
        cudaEventRecord(e0, h->stream);
        if ((r = jac_iterate(h, trial_iters))) return r;
        cudaEventRecord(e1, h->stream);
        if ((r = read_status(h))) return r;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *per = (double)ms / trial_iters;
        return JAC_OK;
    };
    for (int wi = 0; wi < 3 && !rc; ++wi)
        for (int di = 0; di < 4 && !rc; ++di) {
            const int zd = depths[di];
            if (zd != 0 && zd >= max_bz) continue;
            if ((rc = jac_set_tile(h, widths[wi], zd))) break;
            double per = 0.0;
            if ((rc = time_it(&per))) break;
            if (best.n_trials < 16) {
                best.trial_tile_w[best.n_trials] = widths[wi];
                best.trial_zdepth[best.n_trials] = zd;
                best.trial_ms_per_iter[best.n_trials] = per;
            }
            best.n_trials += 1;
            if (per < best.ms_per_iter) {
                best.ms_per_iter = per;
                best.tile_w = widths[wi];
                best.zdepth = zd;
            }
        }
    if (!rc && best.tile_w) rc = jac_set_tile(h, best.tile_w, best.zdepth);
    best.ms_per_iter_classes = best.ms_per_iter;
    // block-width classes, largest (most cells) first
    std::vector<std::pair<int64_t, int32_t>> cls;  // (cells, bx)
    for (const BlockDesc& d : h->hdesc) {
        const int64_t cells = (int64_t)d.ext[0] * d.ext[1] * d.ext[2];
        auto it = std::find_if(cls.begin(), cls.end(),
                               [&](const std::pair<int64_t, int32_t>& c) { return c.second == d.ext[0]; });
        if (it == cls.end()) cls.emplace_back(cells, d.ext[0]);
        else it->first += cells;
    }
    std::sort(cls.begin(), cls.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    if (!rc && cls.size() > 1) {
        double base = 0.0;
        rc = time_it(&base);
        for (size_t c = 0; c < cls.size() && c < 16 && !rc; ++c) {
            const int32_t bx = cls[c].second;
            int32_t keep = best.tile_w;
            for (int wi = 0; wi < 3 && !rc; ++wi) {
                if (widths[wi] == best.tile_w) continue;
                if ((rc = jac_set_tile_class(h, bx, widths[wi]))) break;
                double per = 0.0;
                if ((rc = time_it(&per))) break;
                best.n_trials += 1;
                if (per < base) {
                    base = per;
                    keep = widths[wi];
                }
            }
            if (!rc) rc = jac_set_tile_class(h, bx, keep == best.tile_w ? 0 : keep);
            best.class_block_x[best.n_classes] = bx;
            best.class_tile_w[best.n_classes] = keep;
            best.n_classes += 1;
        }
        best.ms_per_iter_classes = base;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(h->pool, snap, bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaFreeAsync(snap, h->stream);
    h->parity = parity0;
    h->iters = iters0;
    if (rc) return rc;
    if ((rc = forget_unit_frames(h))) return rc;  // the bounds describe the trials' data
    CU(cudaStreamSynchronize(h->stream), "autotune sync");
    if (result) *result = best;
    return JAC_OK;
}

int jac_storage_bytes(const int64_t dims[3], int32_t bx, int32_t by, int32_t bz, int32_t dtype, int64_t* bytes)
{
    if (!dims || !bytes) return fail(JAC_EINVAL, "null argument");
    if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256) return fail(JAC_EINVAL, "bad block dims");
    if (dtype != JAC_F64 && dtype != JAC_F32) return fail(JAC_EINVAL, "bad dtype");
    jac_ctx tmp;
    tmp.req_block[0] = bx;
    tmp.req_block[1] = by;
    tmp.req_block[2] = bz;
    tmp.dtype = dtype;
    tmp.esize = dtype == JAC_F32 ? 4 : 8;
    Instance I;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 30)) return fail(JAC_EINVAL, "bad grid dims");
        I.dims[a] = dims[a];
    }
    *bytes = (instance_geometry(&tmp, I) + 255) / 256 * 256;
    return JAC_OK;
}

int jac_create_pool(jac_ctx** out, int32_t dtype, int64_t capacity_bytes, int32_t max_grids, int32_t bx, int32_t by,
                    int32_t bz, void* stream)
{
    if (!out) return fail(JAC_EINVAL, "null output pointer");
    *out = nullptr;
    if (dtype != JAC_F64 && dtype != JAC_F32) return fail(JAC_EINVAL, "dtype must be JAC_F64 or JAC_F32");
    if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256)
        return fail(JAC_EINVAL, "block dims must be in [1, 256]");
    if (capacity_bytes < 256 || max_grids < 1 || max_grids > (1 << 20)) return fail(JAC_EINVAL, "bad pool size");
    jac_ctx* h = new jac_ctx();
    h->req_block[0] = bx;
    h->req_block[1] = by;
    h->req_block[2] = bz;
    h->dtype = dtype;
    h->esize = dtype == JAC_F32 ? 4 : 8;
    h->arith = dtype == JAC_F32 ? JAC_ARITH_SEQ : JAC_ARITH_EXACT;
    h->max_slots = max_grids;
    h->is_pool = true;
    int rc = open_ctx(h, stream);
    void* pool = nullptr;
    if (!rc) rc = dev_alloc(h, (size_t)capacity_bytes, &pool);
    if (!rc) {
        h->own_arena.init(pool, capacity_bytes);
        h->arena = &h->own_arena;
        h->pool = pool;
        rc = refresh(h);
    }
    if (!rc) rc = sync_stream(h);
    if (rc) {
        std::string msg = g_last_error;
        jac_destroy(h);
        g_last_error = msg;
        return rc;
    }
    *out = h;
    return JAC_OK;
}

int jac_pool_add(jac_ctx* h, const int64_t dims[3], const double bc[6], int32_t* slot)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (!h->is_pool) return fail(JAC_ESTATE, "grids can be added to pools only");
    if (!dims || !bc || !slot) return fail(JAC_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 30)) return fail(JAC_EINVAL, "grid dims must be in [1, 2^30]");
    for (int f = 0; f < 6; ++f)
        if (!value_ok(bc[f], h->dtype)) return fail(JAC_EINVAL, "boundary value %d not finite or out of range", f);
    return add_instance(h, dims, bc, slot);
}

int jac_pool_remove(jac_ctx* h, int32_t slot)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (!h->is_pool) return fail(JAC_ESTATE, "grids can be removed from pools only");
    return remove_instance(h, slot);
}

int jac_pool_usage(jac_ctx* h, int64_t* used_bytes, int64_t* capacity_bytes, int32_t* grids)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (used_bytes) *used_bytes = h->arena ? h->arena->used : 0;
    if (capacity_bytes) *capacity_bytes = h->arena ? h->arena->capacity : 0;
    if (grids) *grids = h->n_active();
    return JAC_OK;
}

int jac_set_wait_limit_ns(jac_ctx* h, int64_t ns)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (ns < 1000) return fail(JAC_EINVAL, "wait limit must be >= 1000 ns");
    h->wait_ns = ns;
    return JAC_OK;
}

int jac_debug_withhold_progress(jac_ctx* h, int32_t block, int64_t after_iter)
{
    int rc = check_ctx(h);
    if (rc) return rc;
    if (block >= (int32_t)h->hdesc.size()) return fail(JAC_EINVAL, "block out of range");
    h->hold_block = block < 0 ? -1 : block;
    h->hold_after = after_iter;
    return JAC_OK;
}


// ====================================================================== server

}  // extern "C"

#include <chrono>
#include <deque>

struct ServeReq {
    int64_t id = 0;
    int64_t dims[3] = {0, 0, 0};
    int32_t dtype = JAC_F64;
    double bc[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> init, result;
    double tol = 0.0;
    int64_t max_iters = 0;
    int64_t iters = 0;
    double residual = 0.0;
    int32_t slot = -1;
    int32_t state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct jac_server {
    int device = 0;
    Arena arena;
    void* base = nullptr;
    size_t base_bytes = 0;
    jac_ctx* pool[2] = {nullptr, nullptr};  // binary64, binary32
    cudaStream_t stream[2] = {nullptr, nullptr};
    double* hres[2] = {nullptr, nullptr};  // pinned per-slot residuals
    int32_t max_active = 0, bx = 64, by = 64, bz = 64, chunk = 50;
    std::deque<int64_t> queue;
    std::map<int64_t, ServeReq> reqs;
    std::deque<int64_t> finished;
    int64_t next_id = 1;
    int32_t running = 0;
    int64_t cell_updates = 0;
    std::chrono::steady_clock::time_point t0;
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

extern "C" {

int jac_server_destroy(jac_server* s)
{
    if (!s) return JAC_OK;
    cudaSetDevice(s->device);
    for (int d = 0; d < 2; ++d) {
        if (s->pool[d]) jac_destroy(s->pool[d]);
        if (s->stream[d]) {
            cudaStreamSynchronize(s->stream[d]);
            cudaStreamDestroy(s->stream[d]);
        }
        if (s->hres[d]) cudaFreeHost(s->hres[d]);
    }
    if (s->base) cudaFree(s->base);
    delete s;
    return JAC_OK;
}

int jac_server_create(jac_server** out, int64_t budget_bytes, int32_t max_active, int32_t bx, int32_t by, int32_t bz,
                      int32_t chunk_iters)
{
    if (!out) return fail(JAC_EINVAL, "null output pointer");
    *out = nullptr;
    if (budget_bytes < 4096 || max_active < 1 || max_active > 65536 || chunk_iters < 1)
        return fail(JAC_EINVAL, "bad server parameters");
    if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256) return fail(JAC_EINVAL, "bad block dims");
    jac_server* s = new jac_server();
    cudaGetDevice(&s->device);
    s->max_active = max_active;
    s->bx = bx;
    s->by = by;
    s->bz = bz;
    s->chunk = chunk_iters;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc(&s->base, (size_t)budget_bytes);
    if (e != cudaSuccess) {
        jac_server_destroy(s);
        return cuda_fail(e, "server arena");
    }
    s->base_bytes = (size_t)budget_bytes;
    s->arena.init(s->base, budget_bytes);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int d = 0; d < 2; ++d) {
        e = cudaStreamCreateWithPriority(&s->stream[d], cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaMallocHost(&s->hres[d], sizeof(double) * (size_t)max_active);
        if (e != cudaSuccess) {
            jac_server_destroy(s);
            return cuda_fail(e, "server streams");
        }
        int rc = create_pool_shared(&s->pool[d], d == 0 ? JAC_F64 : JAC_F32, &s->arena, max_active, bx, by, bz,
                                    (void*)s->stream[d]);
        if (rc) {
            std::string msg = g_last_error;
            jac_server_destroy(s);
            g_last_error = msg;
            return rc;
        }
    }
    *out = s;
    return JAC_OK;
}

int jac_server_submit(jac_server* s, const int64_t dims[3], int32_t dtype, const double bc[6], const double* init,
                      double tol, int64_t max_iters, int64_t* req_id)
{
    if (!s || !dims || !bc || !init || !req_id) return fail(JAC_EINVAL, "null argument");
    if (dtype != JAC_F64 && dtype != JAC_F32) return fail(JAC_EINVAL, "bad dtype");
    if (!(tol >= 0.0) || max_iters < 0) return fail(JAC_EINVAL, "bad stopping rule");
    int64_t n = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 30)) return fail(JAC_EINVAL, "bad grid dims");
        n *= dims[a];
    }
    for (int f = 0; f < 6; ++f)
        if (!value_ok(bc[f], dtype)) return fail(JAC_EINVAL, "boundary value %d not finite or out of range", f);
    for (int64_t q = 0; q < n; ++q)
        if (!value_ok(init[q], dtype)) return fail(JAC_EINVAL, "value at %lld not finite or out of range", (long long)q);
    int64_t bytes = 0;
    int rc = jac_storage_bytes(dims, s->bx, s->by, s->bz, dtype, &bytes);
    if (rc) return rc;
    if (bytes > s->arena.capacity) return fail(JAC_EBUDGET, "grid of %lld bytes exceeds the budget", (long long)bytes);
    ServeReq r;
    r.id = s->next_id++;
    for (int a = 0; a < 3; ++a) r.dims[a] = dims[a];
    for (int f = 0; f < 6; ++f) r.bc[f] = bc[f];
    r.dtype = dtype;
    r.init.assign(init, init + n);
    r.tol = tol;
    r.max_iters = max_iters;
    r.t_submit = s->now();
    s->queue.push_back(r.id);
    *req_id = r.id;
    s->reqs.emplace(r.id, std::move(r));
    return JAC_OK;
}

// One round: admit queued requests (first come, first served) while a slot
// and room in the arena are free, advance every resident grid by one chunk
// (binary64 and binary32 pools on their own streams, so their launches
// overlap), read the per-grid binary64 residuals, and retire every grid
// whose residual fell below its tolerance or that reached its iteration cap.
int jac_server_step(jac_server* s, jac_server_stats_t* stats)
{
    if (!s) return fail(JAC_EINVAL, "null server");
    cudaSetDevice(s->device);
    int rc;
    while (!s->queue.empty() && s->running < s->max_active) {
        ServeReq& r = s->reqs[s->queue.front()];
        const int d = r.dtype == JAC_F32 ? 1 : 0;
        int32_t slot = -1;
        rc = jac_pool_add(s->pool[d], r.dims, r.bc, &slot);
        if (rc == JAC_EBUDGET) break;  // wait until a running grid frees its region
        if (!rc) rc = jac_write_instance(s->pool[d], slot, r.init.data(), r.init.size());
        s->queue.pop_front();
        if (rc) {
            r.state = 3;
            r.t_done = s->now();
            s->finished.push_back(r.id);
            if (slot >= 0) jac_pool_remove(s->pool[d], slot);
            continue;
        }
        r.slot = slot;
        r.state = 1;
        r.t_admit = s->now();
        r.init.clear();
        r.init.shrink_to_fit();
        s->running += 1;
    }
    bool any[2] = {false, false};
    for (int d = 0; d < 2; ++d) {
        jac_ctx* h = s->pool[d];
        if (h->n_active() == 0) continue;
        any[d] = true;
        if ((rc = jac_iterate(h, s->chunk))) return rc;
        if ((rc = jac_residual_instances_device(h, h->dres_inst))) return rc;
        CU(cudaMemcpyAsync(s->hres[d], h->dres_inst, sizeof(double) * h->inst.size(), cudaMemcpyDeviceToHost,
                           h->stream),
           "copy residuals");
    }
    for (int d = 0; d < 2; ++d)
        if (any[d] && (rc = jac_sync(s->pool[d]))) return rc;
    int32_t done_now = 0;
    for (auto& kv : s->reqs) {
        ServeReq& r = kv.second;
        if (r.state != 1) continue;
        const int d = r.dtype == JAC_F32 ? 1 : 0;
        r.iters += s->chunk;
        r.residual = s->hres[d][r.slot];
        s->cell_updates += r.dims[0] * r.dims[1] * r.dims[2] * (int64_t)s->chunk;
        if (r.residual < r.tol || r.iters >= r.max_iters) {
            r.result.resize((size_t)(r.dims[0] * r.dims[1] * r.dims[2]));
            rc = jac_read_instance(s->pool[d], r.slot, r.result.data(), r.result.size());
            jac_pool_remove(s->pool[d], r.slot);
            r.state = rc ? 3 : 2;
            r.t_done = s->now();
            s->running -= 1;
            s->finished.push_back(r.id);
            done_now += 1;
        }
    }
    if (stats) {
        stats->running = s->running;
        stats->queued = (int32_t)s->queue.size();
        stats->finished_now = done_now;
        stats->cell_updates = s->cell_updates;
        stats->used_bytes = s->arena.used;
        stats->budget_bytes = s->arena.capacity;
    }
    return JAC_OK;
}

int jac_server_poll(jac_server* s, jac_request_t* out)
{
    if (!s || !out) return fail(JAC_EINVAL, "null argument");
    if (s->finished.empty()) return JAC_ESTATE;
    const ServeReq& r = s->reqs[s->finished.front()];
    s->finished.pop_front();
    out->id = r.id;
    out->iterations = r.iters;
    out->residual = r.residual;
    out->t_submit = r.t_submit;
    out->t_admit = r.t_admit;
    out->t_done = r.t_done;
    out->status = r.state == 2 ? JAC_OK : JAC_ECUDA;
    return JAC_OK;
}

int jac_server_result(jac_server* s, int64_t req_id, double* host_out, size_t n_cells)
{
    if (!s) return fail(JAC_EINVAL, "null server");
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || it->second.state < 2) return fail(JAC_ESTATE, "request %lld not finished", (long long)req_id);
    ServeReq& r = it->second;
    if (host_out) {
        if (n_cells != r.result.size()) return fail(JAC_EINVAL, "n_cells %zu != %zu", n_cells, r.result.size());
        memcpy(host_out, r.result.data(), n_cells * sizeof(double));
    }
    s->reqs.erase(it);  // the result is handed over once
    return JAC_OK;
}

int jac_server_now(jac_server* s, double* seconds)
{
    if (!s || !seconds) return fail(JAC_EINVAL, "null argument");
    *seconds = s->now();
    return JAC_OK;
}

}  // extern "C"
