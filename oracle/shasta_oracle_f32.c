/*
 * shasta_oracle_f32.c -- the plain oracle evaluated in single precision.
 *
 * TEST INFRASTRUCTURE, like shasta_oracle.c: only the test suite and the
 * script that writes the stored sensitivity figures may build, load or call
 * it; it shares no code with the CUDA library.
 *
 * The paper's own GPU implementation keeps every quantity in single
 * precision (Sec. 3.1.4) and is compared in Sec. 4 with a double-precision
 * code.  This unit compiles the unchanged oracle source with every double
 * replaced by float (and, through -fsingle-precision-constant, every
 * literal constant in single precision), so each operation of the plain
 * algorithm rounds to single precision in the oracle's order.  It is not a
 * second reference: the tests use the distance between this build and the
 * double-precision oracle as the size of the error that single-precision
 * rounding alone produces, where the flow amplifies rounding too much for a
 * single-precision result to be held to a fixed tolerance.
 *
 * Build: gcc -O2 -ffp-contract=off -fsingle-precision-constant.  The math
 * functions map to their single-precision forms; square root, floor,
 * minimum, maximum and absolute value are exact or correctly rounded in
 * both forms.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define double float
#define sqrt sqrtf
#define fabs fabsf
#define fmin fminf
#define fmax fmaxf
#define floor floorf

#include "shasta_oracle.c"
