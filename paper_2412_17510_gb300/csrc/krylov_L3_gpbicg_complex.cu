// krylov_L3_gpbicg_complex.cu -- triple-double (L = 3) GPBiCG, complex data.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<3, true, mpkry::KRY_GPBICG>;
