/* Internal helpers of the oracle (test infrastructure only). */
#ifndef OR_COMMON_H
#define OR_COMMON_H
#include "oracle.h"

extern int or_count_on;
extern long long or_count;
/* add n floating-point operations (add, sub, mul, div, exp, sqrt each count 1) */
#define OR_FLOPS(n) do { if (or_count_on) or_count += (n); } while (0)
/* branch signature: a running hash of the BESSER control-point branches taken
   (in call order) while recording is on; two evaluations of the same map that
   take the same branches everywhere have the same signature */
extern int or_sig_on;
extern unsigned long long or_sig;
#define OR_BRANCH(b) do { if (or_sig_on) { or_sig ^= (unsigned long long)(b) + 1ULL; or_sig *= 1099511628211ULL; } } while (0)

#endif
