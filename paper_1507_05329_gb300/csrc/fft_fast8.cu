// Row and pencil FFT kernels for plans whose largest radix is 8.
#define COLA_MAXR 8
#define COLA_PART_MAIN 1
#define COLA_PART_GREEN 0
#include "fft_fast.inc"
