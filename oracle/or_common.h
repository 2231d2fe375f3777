/* Internal helpers of the oracle (test infrastructure only). */
#ifndef OR_COMMON_H
#define OR_COMMON_H
#include "oracle.h"

extern int or_count_on;
extern long long or_count;
/* add n floating-point operations (add, sub, mul, div, exp, sqrt each count 1) */
#define OR_FLOPS(n) do { if (or_count_on) or_count += (n); } while (0)

#endif
