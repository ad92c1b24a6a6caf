// Kernels of libhom in complex128 (FP64 arithmetic).
#define HOM_T double
#define HOM_WIDE 0
#include "hom_kern.inc"
