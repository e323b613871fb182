// krylov_L4_cgs.cu -- quad-double (L = 4) CGS, real and complex.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<4, false, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<4, true, mpkry::KRY_CGS>;
