// In-place kinetic passes of libhom in complex64 (single and double).
#define HOM_T float
#define HOM_WIDE 1
#define HOM_PART 1
#include "hom_kern.inc"
