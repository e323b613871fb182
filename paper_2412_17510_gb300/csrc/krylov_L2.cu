// krylov_L2.cu -- double-double (L = 2): CG and the vector operations, and the nonsymmetric methods.
#include "krylov_impl.cuh"

template struct mpkry::KrylovOps<2>;
template struct mpkry::KrylovSolve<2, false, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<2, true, mpkry::KRY_BICGSTAB>;
template struct mpkry::KrylovSolve<2, false, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<2, true, mpkry::KRY_BICG>;
template struct mpkry::KrylovSolve<2, false, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<2, true, mpkry::KRY_CGS>;
template struct mpkry::KrylovSolve<2, false, mpkry::KRY_GPBICG>;
template struct mpkry::KrylovSolve<2, true, mpkry::KRY_GPBICG>;
