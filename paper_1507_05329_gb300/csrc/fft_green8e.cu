// Fused Green-function FFT kernels with 8 elements per thread, plans whose largest radix is 8.
#define COLA_MAXR 8
#define COLA_PART_MAIN 0
#define COLA_PART_GREEN 1
#define COLA_GREEN_EPT 8
#include "fft_fast.inc"
