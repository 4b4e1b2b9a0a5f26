/* ORACLE (test infrastructure only): float and double instantiations of the particle stages. */
#include "oracle_internal.h"

#define PREAL float
#define PFN(n) n##_f32
#define PLOG or_logf
#define PSQRT sqrtf
#define PSINCOS or_sincos2pif
#define PUNIF or_uniforms_f
#define PLRINT llrintf
#include "oracle_particles.inc"
#undef PREAL
#undef PFN
#undef PLOG
#undef PSQRT
#undef PSINCOS
#undef PUNIF
#undef PLRINT

#define PREAL double
#define PFN(n) n##_f64
#define PLOG or_logd
#define PSQRT sqrt
#define PSINCOS or_sincos2pid
#define PUNIF or_uniforms_d
#define PLRINT llrint
#include "oracle_particles.inc"
