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
