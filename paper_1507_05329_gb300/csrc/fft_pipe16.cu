// Persistent cp.async-pipelined strided FFT passes for plans whose largest radix is 16.
#define COLA_MAXR 16
#define COLA_PART_MAIN 0
#define COLA_PART_GREEN 0
#define COLA_PART_PIPE 1
#include "fft_fast.inc"
