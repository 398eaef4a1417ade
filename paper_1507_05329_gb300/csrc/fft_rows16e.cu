// Row (R2C / C2R) FFT kernels with 8 elements per thread, plans whose largest radix is 16.
#define COLA_MAXR 16
#define COLA_PART_MAIN 0
#define COLA_PART_GREEN 0
#define COLA_PART_ROWS 1
#define COLA_ROW_EPT 8
#include "fft_fast.inc"
