// krylov_L3_bicg.cu -- triple-double (L = 3) BiCG, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<3, false, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<3, true, mpkry::KRY_BICG>;
