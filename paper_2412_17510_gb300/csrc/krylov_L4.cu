// krylov_L4.cu -- quad-double (L = 4): CG and the vector operations.
#include "krylov_impl.cuh"

template struct mpkry::KrylovOps<4>;
