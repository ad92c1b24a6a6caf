// In-place kinetic passes of libhom in complex128 (single and double).
#define HOM_T double
#define HOM_WIDE 0
#define HOM_PART 1
#include "hom_kern.inc"
