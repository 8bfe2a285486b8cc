// Host build of the library's integer exact-mean / exact-Laplacian routines
// (paper_2202_11819_gb300/csrc/arith.cuh), so their bit logic can be checked
// against the oracle on a CPU. Test infrastructure only.
#include "arith.cuh"

extern "C" double host_mean7_exact(const double* v)
{
    return jac::mean7_exact(v[0], v[1], v[2], v[3], v[4], v[5], v[6]);
}

extern "C" double host_laplacian_exact(double c, const double* nb)
{
    return jac::laplacian_exact(c, nb[0], nb[1], nb[2], nb[3], nb[4], nb[5]);
}

extern "C" int host_frame_mean7(const double* v, int eref, double* out)
{
    using namespace jac::frame;
    W96 w[7];
    for (int i = 0; i < 7; ++i) w[i] = of(v[i], eref);
    return mean7(w[0], w[1], w[2], w[3], w[4], w[5], w[6], eref, *out) ? 1 : 0;
}

extern "C" int host_frame_laplacian(double c, const double* nb, int eref, double* out)
{
    using namespace jac::frame;
    return laplacian(of(c, eref), of(nb[0], eref), of(nb[1], eref), of(nb[2], eref), of(nb[3], eref),
                     of(nb[4], eref), of(nb[5], eref), eref, *out)
               ? 1
               : 0;
}

// 96-bit frame sum of seven values (for checks of the carry chain).
extern "C" void host_frame_sum7(const double* v, int eref, uint32_t* s)
{
    using namespace jac::frame;
    W96 w[7];
    for (int i = 0; i < 7; ++i) w[i] = of(v[i], eref);
    sum7(w[0], w[1], w[2], w[3], w[4], w[5], w[6], s[0], s[1], s[2]);
}

// The top-binade fast path of the mean: 1 and the mean when the frame sum of
// the seven values qualifies (sum_in_top, eref >= 7), else 0.
extern "C" int host_frame_mean7_top(const double* v, int eref, double* out)
{
    using namespace jac::frame;
    W96 w[7];
    for (int i = 0; i < 7; ++i) w[i] = of(v[i], eref);
    uint32_t s0, s1, s2;
    sum7(w[0], w[1], w[2], w[3], w[4], w[5], w[6], s0, s1, s2);
    if (eref < 7 || !sum_in_top(s2)) return 0;
    *out = mean7_top(s0, s1, s2, (uint32_t)(eref - 1081) << 20);
    return 1;
}

// The binary64 division by 7 of the sequential rule: 1 and RN(s / 7) when
// its integer path applies, else 0.
// The integer addition of the sequential rule: 1 and RN(a + b) when it
// applies, else 0.
extern "C" int host_dadd_nonneg(double a, double b, double* out)
{
    return jac::dadd_nonneg(a, b, *out) ? 1 : 0;
}

extern "C" int host_div7d(double s, double* out)
{
    return jac::div7d(s, *out) ? 1 : 0;
}

// The binary32 residual's 64-bit frame: a value's frame integer (and
// whether it lies in the window), and the sum of squares of n integers over
// 192 bits rounded once and scaled by 2^scale.
extern "C" int host_of32(float v, int eref32, long long* w)
{
    bool ok;
    *w = jac::frame::of32(v, eref32, ok);
    return ok ? 1 : 0;
}

extern "C" double host_sum_squares(const long long* L, int n, int scale)
{
    uint64_t a0 = 0, a1 = 0, a2 = 0;
    for (int i = 0; i < n; ++i) jac::frame::add_square(L[i], a0, a1, a2);
    return jac::frame::u192_to_double_scaled(a0, a1, a2, scale);
}

// The 96-bit frame value of v (four words, the last one padding).
extern "C" void host_frame_of(double v, int eref, uint32_t* w)
{
    const jac::frame::W96 r = jac::frame::of(v, eref);
    w[0] = r.w0;
    w[1] = r.w1;
    w[2] = r.w2;
    w[3] = r.w3;
}

// The 64-bit frame: a value's frame integer and whether it lies in the
// window (zero_ok: the zero-accepting form), and the same integer widened
// to the 96-bit frame.
extern "C" int host_nframe_of(double v, int eref, int zero_ok, unsigned long long* w)
{
    bool ok;
    const uint32_t e = jac::nframe::elo_hi(eref);
    *w = zero_ok ? jac::nframe::of0(v, e, ok) : jac::nframe::of(v, e, ok);
    return ok ? 1 : 0;
}

extern "C" void host_nframe_widen(unsigned long long w, uint32_t* out)
{
    const jac::frame::W96 r = jac::nframe::widen(w);
    out[0] = r.w0;
    out[1] = r.w1;
    out[2] = r.w2;
}

// The 64-bit frame mean as the engine forms it: the cell v[0] through `of`,
// its six neighbours through `of0`, one 64-bit sum, then mean7. Returns 0
// (out unset) when the engine would take the 96-bit frame instead.
extern "C" int host_nframe_mean7(const double* v, int eref, double* out)
{
    using namespace jac::nframe;
    if (eref < 13) return 0;
    const uint32_t e = elo_hi(eref);
    bool ok;
    uint64_t S = of(v[0], e, ok);
    if (!ok) return 0;
    for (int i = 1; i < 7; ++i) {
        S += of0(v[i], e, ok);
        if (!ok) return 0;
    }
    *out = mean7(S, scale_hi(eref));
    return 1;
}

// ---- binary32 residual in split words (r32), for a grid whose largest
// binary32 exponent field is f.

// The split of v: 1 when exact; hg = (H, G), the offsets of the two bit
// patterns from those of C1 and C2. -1 when the frame is out of range.
extern "C" int host_r32_split(float v, int f, int32_t* hg)
{
    using namespace jac::r32;
    const int E = frame_E(f);
    if (!frame_ok(E)) return -1;
    const float c1 = c15(E + 1), c2 = c15(E - 22);
    bool inexact = false;
    const Split s = split(v, c1, c2, inexact);
    hg[0] = (int32_t)(s.h - fbits(c1));
    hg[1] = (int32_t)(s.g - fbits(c2));
    return inexact ? 0 : 1;
}

// The two parts of L for one cell (v = c, xm, xp, ym, yp, zm, zp):
// L = (LH 2^23 + LG) 2^(E - 45). Returns as host_r32_split.
extern "C" int host_r32_laplacian(const float* v, int f, int32_t* lhg)
{
    using namespace jac::r32;
    const int E = frame_E(f);
    if (!frame_ok(E)) return -1;
    const float c1 = c15(E + 1), c2 = c15(E - 22);
    bool inexact = false;
    Split s[7];
    for (int j = 0; j < 7; ++j) s[j] = split(v[j], c1, c2, inexact);
    lhg[0] = lpart(s[0].h, s[1].h, s[2].h, s[3].h, s[4].h, s[5].h, s[6].h);
    lhg[1] = lpart(s[0].g, s[1].g, s[2].g, s[3].g, s[4].g, s[5].g, s[6].g);
    return inexact ? 0 : 1;
}

// The sum of L^2 over n cells as one engine thread forms it (the three
// 64-bit sums in acc3), combined in 128 bits and rounded once (out).
// Returns as host_r32_split.
extern "C" int host_r32_sum_squares(const float* v, int n, int f, int64_t* acc3, double* out)
{
    using namespace jac::r32;
    const int E = frame_E(f);
    if (!frame_ok(E)) return -1;
    const float c1 = c15(E + 1), c2 = c15(E - 22);
    bool inexact = false;
    Acc a{0, 0, 0};
    for (int i = 0; i < n; ++i) {
        Split s[7];
        for (int j = 0; j < 7; ++j) s[j] = split(v[7 * i + j], c1, c2, inexact);
        add_square(lpart(s[0].h, s[1].h, s[2].h, s[3].h, s[4].h, s[5].h, s[6].h),
                   lpart(s[0].g, s[1].g, s[2].g, s[3].g, s[4].g, s[5].g, s[6].g), a);
    }
    acc3[0] = a.a;
    acc3[1] = a.b;
    acc3[2] = a.c;
    uint64_t lo, hi;
    combine(a, lo, hi);
    *out = jac::frame::u192_to_double_scaled(lo, hi, 0u, 2 * E - 90);
    return inexact ? 0 : 1;
}

// S = a 2^46 + b 2^24 + c in 128 bits (lohi = low word, high word).
extern "C" void host_r32_combine(const int64_t* abc, uint64_t* lohi)
{
    jac::r32::Acc a{abc[0], abc[1], abc[2]};
    jac::r32::combine(a, lohi[0], lohi[1]);
}

// The binary64 residual's integer form in the 64-bit frame of eref: over n
// cells (c, xm, xp, ym, yp, zm, zp), L = S - 7c from the frame integers
// (S the sum of the seven), L^2 summed in 192 bits and rounded once, scaled
// by 2^(2 (eref - 1084)). 1 and the sum when every value lies in the frame
// (neighbours may be +0), else 0.
extern "C" int host_nframe_residual(const double* v, int n, int eref, double* out)
{
    using namespace jac;
    const uint32_t elo = nframe::elo_hi(eref);
    uint64_t q0 = 0u, q1 = 0u, q2 = 0u;
    for (int i = 0; i < n; ++i) {
        const double* w = v + 7 * i;
        bool ok = true, g;
        const uint64_t c = nframe::of(w[0], elo, g);
        ok = ok && g;
        uint64_t S = c;
        for (int j = 1; j < 7; ++j) {
            S += nframe::of0(w[j], elo, g);
            ok = ok && g;
        }
        if (!ok) return 0;
        nframe::add_laplacian_square(S, c, q0, q1, q2);
    }
    *out = frame::u192_to_double_scaled(q0, q1, q2, 2 * (eref - 1084));
    return 1;
}
