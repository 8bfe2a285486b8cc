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
