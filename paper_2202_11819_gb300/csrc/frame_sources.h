// Frame sources of the work units of the exact mean (host code).
//
// A tile of the correctly rounded mean takes its fixed-point frame from the
// exponent bounds that the previous iteration's units wrote for the values
// it reads. The frame sources of a unit are those units: the units its
// haloed box overlaps in its own block (the x and y halo columns and rows,
// the planes below and above its z range), and in each neighbouring block
// the units of the face column, row or plane next to it. The list may hold
// more than the tile reads (corner cells, whole face rows), never less.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include "jac_common.cuh"

namespace jac {

// A unit with more sources than this gets no list (fsn = -1): the engine
// then takes the bounds of every unit of its block and its neighbours.
constexpr int kMaxFrameSources = 256;

// Sets each unit's fs0, fsn and appends its sources to src. rows(tw) is the
// number of tile rows of a unit tw columns wide; each block's units are
// desc[b].u0 .. desc[b].u0 + desc[b].ntiles - 1.
template <typename Rows>
inline void build_frame_sources(std::vector<TileUnit>& units, const std::vector<BlockDesc>& desc, Rows rows,
                                std::vector<int32_t>& src)
{
    src.clear();
    // units of block nb overlapping columns [xa, xb], rows [ya, yb], planes [za, zb] (inclusive)
    auto add = [&](int32_t nb, int xa, int xb, int ya, int yb, int za, int zb) {
        if (nb < 0 || xa > xb || ya > yb || za > zb) return;
        const BlockDesc& n = desc[nb];
        for (int32_t v = n.u0; v >= 0 && v < n.u0 + n.ntiles; ++v) {
            const TileUnit& w = units[v];
            const int th = rows(w.tw);
            if (w.x0 <= xb && w.x0 + w.tw - 1 >= xa && w.y0 <= yb && w.y0 + th - 1 >= ya && w.z0 <= zb &&
                w.z1 - 1 >= za)
                src.push_back(v);
        }
    };
    for (size_t i = 0; i < units.size(); ++i) {
        TileUnit& u = units[i];
        const BlockDesc& d = desc[u.block];
        const int bx = d.ext[0], by = d.ext[1], bz = d.ext[2], th = rows(u.tw);
        const int x1 = std::min<int>(u.x0 + u.tw, bx) - 1, y1 = std::min<int>(u.y0 + th, by) - 1, z1 = u.z1 - 1;
        const size_t start = src.size();
        add(u.block, std::max(0, u.x0 - 1), std::min(bx - 1, x1 + 1), std::max(0, u.y0 - 1), std::min(by - 1, y1 + 1),
            std::max(0, u.z0 - 1), std::min(bz - 1, z1 + 1));
        if (u.x0 == 0 && d.nbr[0] >= 0)
            add(d.nbr[0], desc[d.nbr[0]].ext[0] - 1, desc[d.nbr[0]].ext[0] - 1, u.y0, y1, u.z0, z1);
        if (x1 == bx - 1 && d.nbr[1] >= 0) add(d.nbr[1], 0, 0, u.y0, y1, u.z0, z1);
        if (u.y0 == 0 && d.nbr[2] >= 0)
            add(d.nbr[2], u.x0, x1, desc[d.nbr[2]].ext[1] - 1, desc[d.nbr[2]].ext[1] - 1, u.z0, z1);
        if (y1 == by - 1 && d.nbr[3] >= 0) add(d.nbr[3], u.x0, x1, 0, 0, u.z0, z1);
        if (u.z0 == 0 && d.nbr[4] >= 0)
            add(d.nbr[4], u.x0, x1, u.y0, y1, desc[d.nbr[4]].ext[2] - 1, desc[d.nbr[4]].ext[2] - 1);
        if (z1 == bz - 1 && d.nbr[5] >= 0) add(d.nbr[5], u.x0, x1, u.y0, y1, 0, 0);
        u.fs0 = (int32_t)start;
        u.fsn = (int32_t)(src.size() - start);
        if (u.fsn > kMaxFrameSources) {
            src.resize(start);
            u.fsn = -1;
        }
    }
}

}  // namespace jac
