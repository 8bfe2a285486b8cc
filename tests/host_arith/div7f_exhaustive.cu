// Every finite binary32 value s: the library's div7f(s) against the
// correctly rounded quotient RN(s / 7). The reference is (float)((double)s /
// 7.0): s / 7 is either exact in binary32 or has a binary expansion that
// repeats with period 3 past the 24th bit, so the double quotient never sits
// on a binary32 rounding boundary it was not already on and rounding twice
// gives the correctly rounded result. Test infrastructure only.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "arith.cuh"

int main()
{
    long bad = 0, checked = 0;
#pragma omp parallel for reduction(+ : bad, checked) schedule(static)
    for (long i = 0; i <= 0xFFFFFFFFL; ++i) {
        const uint32_t b = (uint32_t)i;
        float x;
        memcpy(&x, &b, 4);
        if (!std::isfinite(x)) continue;
        const float want = (float)((double)x / 7.0);
        const float got = jac::div7f(x);
        ++checked;
        if (memcmp(&got, &want, 4) != 0) ++bad;
    }
    printf("checked=%ld bad=%ld\n", checked, bad);
    return bad != 0;
}
