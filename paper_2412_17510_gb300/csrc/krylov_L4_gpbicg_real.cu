// krylov_L4_gpbicg_real.cu -- quad-double (L = 4) GPBiCG, real data.
#include "krylov_impl.cuh"

template struct mpkry::KrylovSolve<4, false, mpkry::KRY_GPBICG>;
