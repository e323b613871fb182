// krylov_L4_bicg.cu -- quad-double (L = 4) BiCG, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<4, false, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<4, true, mpkry::KRY_BICG>;
