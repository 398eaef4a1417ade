// Fused Green-function FFT kernels for plans whose largest radix is 16.
#define COLA_MAXR 16
#define COLA_PART_MAIN 0
#define COLA_PART_GREEN 1
#include "fft_fast.inc"
