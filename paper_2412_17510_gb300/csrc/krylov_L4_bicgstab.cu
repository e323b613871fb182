// krylov_L4_bicgstab.cu -- quad-double (L = 4) BiCGSTAB, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<4, false, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<4, true, mpkry::KRY_BICGSTAB>;
