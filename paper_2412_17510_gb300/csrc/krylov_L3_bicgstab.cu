// krylov_L3_bicgstab.cu -- triple-double (L = 3) BiCGSTAB, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<3, false, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<3, true, mpkry::KRY_BICGSTAB>;
