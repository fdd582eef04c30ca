/*
 * CPU oracle for the two-stage Hessenberg-triangular reduction (Steel & Vandebril).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline load this library.  It shares no code, header or table with the GPU library.
 *
 * Exported symbols (suffix _d: FP64, suffix _ld: C long double):
 *   oracle_larfg_{d,ld}   Householder reflector (LAPACK dlarfg convention)
 *   oracle_stage0_{d,ld}  QR of B, applied to A and accumulated into Q
 *   oracle_stage1_{d,ld}  Alg. 1, dense (A, triangular B) -> r-HT, reflectors one at a time
 *   oracle_stage2_{d,ld}  Alg. 2, r-HT -> HT, reflectors one at a time
 * Q and Z may be NULL (not accumulated); otherwise they are multiplied from the right
 * (Q := Q Q_stage, Z := Z Z_stage), so passing identities yields the stage's own factors.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared hts_oracle.c -o liboracle.so -lm
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Minimum amount of work (entries touched) before a reflector application is threaded. */
#define PAR_MIN 65536L

#define REAL double
#define FN(name) name##_d
#define SQRT sqrt
#include "hts_oracle_body.inc"
#undef REAL
#undef FN
#undef SQRT

#define REAL long double
#define FN(name) name##_ld
#define SQRT sqrtl
#include "hts_oracle_body.inc"
#undef REAL
#undef FN
#undef SQRT

/* Number of OpenMP threads a parallel region of the oracle uses. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Mantissa digits of long double on this platform (64 on x86-64, 113 on AArch64). */
int oracle_ldbl_mant_dig(void) { return __LDBL_MANT_DIG__; }
