// Row and pencil FFT kernels for plans whose largest radix is 16.
#define COLA_MAXR 16
#define COLA_PART_MAIN 1
#define COLA_PART_GREEN 0
#include "fft_fast.inc"
