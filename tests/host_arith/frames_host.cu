// Host check of the frame-source lists (paper_2202_11819_gb300/csrc/frame_sources.h)
// on synthetic block layouts: every cell a unit's tile reads must belong to
// a unit in its list. Test infrastructure only.
#include <algorithm>
#include <vector>

#include "frame_sources.h"

using namespace jac;

namespace {

// n cells in ceil(n / b) blocks whose sizes differ by at most one, the larger first
void split(int n, int b, std::vector<int>& size, std::vector<int>& org)
{
    const int nb = (n + b - 1) / b, base = n / nb, rem = n % nb;
    size.assign(nb, 0);
    org.assign(nb, 0);
    int o = 0;
    for (int i = 0; i < nb; ++i) {
        size[i] = base + (i < rem ? 1 : 0);
        org[i] = o;
        o += size[i];
    }
}

}  // namespace

// Blocks of b* over a grid of n*, units of tw x th columns over zdepth planes
// (0: the whole block), every split_every-th unit halved in z (0: none);
// drop_last removes the last source of every list that has several (the
// check must then fail). stats: units, reads checked, reads whose unit is
// missing from the list, units without a list, longest list.
extern "C" int host_frame_sources_check(int nx, int ny, int nz, int bx, int by, int bz, int tw, int th, int zdepth,
                                        int split_every, int drop_last, long long* stats)
{
    std::vector<int> sx, ox, sy, oy, sz, oz;
    split(nx, bx, sx, ox);
    split(ny, by, sy, oy);
    split(nz, bz, sz, oz);
    const int NX = (int)sx.size(), NY = (int)sy.size(), NZ = (int)sz.size();
    std::vector<BlockDesc> desc(NX * NY * NZ);
    auto bid = [&](int i, int j, int k) { return i + NX * (j + NY * k); };
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                BlockDesc& d = desc[bid(i, j, k)];
                d = BlockDesc{};
                d.ext[0] = sx[i];
                d.ext[1] = sy[j];
                d.ext[2] = sz[k];
                d.nbr[0] = i > 0 ? bid(i - 1, j, k) : -1;
                d.nbr[1] = i + 1 < NX ? bid(i + 1, j, k) : -1;
                d.nbr[2] = j > 0 ? bid(i, j - 1, k) : -1;
                d.nbr[3] = j + 1 < NY ? bid(i, j + 1, k) : -1;
                d.nbr[4] = k > 0 ? bid(i, j, k - 1) : -1;
                d.nbr[5] = k + 1 < NZ ? bid(i, j, k + 1) : -1;
            }
    std::vector<TileUnit> units;
    int count = 0;
    for (int b = 0; b < (int)desc.size(); ++b) {
        BlockDesc& d = desc[b];
        d.u0 = (int)units.size();
        const int zd = zdepth > 0 ? zdepth : d.ext[2];
        for (int z0 = 0; z0 < d.ext[2]; z0 += zd)
            for (int y0 = 0; y0 < d.ext[1]; y0 += th)
                for (int x0 = 0; x0 < d.ext[0]; x0 += tw) {
                    TileUnit u{};
                    u.block = b;
                    u.x0 = (int16_t)x0;
                    u.y0 = (int16_t)y0;
                    u.z0 = (int16_t)z0;
                    u.z1 = (int16_t)std::min(d.ext[2], z0 + zd);
                    u.tw = (int16_t)tw;
                    ++count;
                    if (split_every > 0 && count % split_every == 0 && u.z1 - u.z0 >= 2) {
                        TileUnit lo = u, hi = u;
                        lo.z1 = hi.z0 = (int16_t)((u.z0 + u.z1) / 2);
                        units.push_back(lo);
                        units.push_back(hi);
                    } else {
                        units.push_back(u);
                    }
                }
        d.ntiles = (int)units.size() - d.u0;
    }
    std::vector<int32_t> src;
    build_frame_sources(units, desc, [th](int) { return th; }, src);
    long long reads = 0, missing = 0, nolist = 0, longest = 0;
    // the unit of block b holding local cell (x, y, z)
    auto unit_of = [&](int b, int x, int y, int z) {
        const BlockDesc& d = desc[b];
        for (int v = d.u0; v < d.u0 + d.ntiles; ++v) {
            const TileUnit& w = units[v];
            if (x >= w.x0 && x < w.x0 + w.tw && y >= w.y0 && y < w.y0 + th && z >= w.z0 && z < w.z1) return v;
        }
        return -1;
    };
    for (size_t i = 0; i < units.size(); ++i) {
        const TileUnit& u = units[i];
        if (u.fsn < 0) {
            ++nolist;
            continue;
        }
        longest = std::max<long long>(longest, u.fsn);
        const int n = (drop_last && u.fsn > 1) ? u.fsn - 1 : u.fsn;
        const BlockDesc& d = desc[u.block];
        const int x1 = std::min<int>(u.x0 + u.tw, d.ext[0]), y1 = std::min<int>(u.y0 + th, d.ext[1]);
        for (int z = u.z0; z < u.z1; ++z)
            for (int y = u.y0; y < y1; ++y)
                for (int x = u.x0; x < x1; ++x) {
                    const int nb6[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                                           {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
                    for (int f = 0; f < 6; ++f) {
                        int cx = nb6[f][0], cy = nb6[f][1], cz = nb6[f][2], b = u.block;
                        const int axis = f / 2;
                        int c[3] = {cx, cy, cz};
                        if (c[axis] < 0 || c[axis] >= d.ext[axis]) {
                            b = d.nbr[f];
                            if (b < 0) continue;  // a Dirichlet ghost
                            c[axis] = c[axis] < 0 ? desc[b].ext[axis] - 1 : 0;
                        }
                        const int v = unit_of(b, c[0], c[1], c[2]);
                        ++reads;
                        bool found = false;
                        for (int s = 0; s < n && !found; ++s) found = src[u.fs0 + s] == v;
                        if (!found) ++missing;
                    }
                }
    }
    stats[0] = (long long)units.size();
    stats[1] = reads;
    stats[2] = missing;
    stats[3] = nolist;
    stats[4] = longest;
    return 0;
}
