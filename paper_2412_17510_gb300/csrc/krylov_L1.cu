// krylov_L1.cu -- binary64 (L = 1): CG and the vector operations, and the nonsymmetric methods.
#include "krylov_impl.cuh"

template struct mpkry::KrylovOps<1>;
template struct mpkry::KrylovSolve<1, false, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<1, true, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<1, false, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<1, true, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<1, false, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<1, true, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<1, false, mpkry::KRY_GPBICG>;
template struct mpkry::KrylovSolve<1, true, mpkry::KRY_GPBICG>;
