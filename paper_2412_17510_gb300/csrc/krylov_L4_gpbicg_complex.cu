// krylov_L4_gpbicg_complex.cu -- quad-double (L = 4) GPBiCG, complex data.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<4, true, mpkry::KRY_GPBICG>;
