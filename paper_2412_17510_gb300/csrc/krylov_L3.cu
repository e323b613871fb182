// krylov_L3.cu -- triple-double (L = 3): CG and the vector operations.
#include "krylov_impl.cuh"

template struct mpkry::KrylovOps<3>;
