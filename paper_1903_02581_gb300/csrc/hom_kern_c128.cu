// Kernels of libhom in complex128 (FP64 arithmetic): the transposing pass
// and every kernel but the in-place passes.
#define HOM_T double
#define HOM_WIDE 0
#define HOM_PART 2
#include "hom_kern.inc"
