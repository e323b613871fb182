// krylov_L3_cgs.cu -- triple-double (L = 3) CGS, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<3, false, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<3, true, mpkry::KRY_CGS>;
