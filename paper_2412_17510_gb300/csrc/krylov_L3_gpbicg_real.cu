// krylov_L3_gpbicg_real.cu -- triple-double (L = 3) GPBiCG, real data.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<3, false, mpkry::KRY_GPBICG>;
