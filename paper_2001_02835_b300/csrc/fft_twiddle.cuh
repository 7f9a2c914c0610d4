// Twiddle table w^n = exp(2 pi i n / NSPT_FFT_MAX_LEN), n = 0..NSPT_FFT_MAX_LEN-1,
// generated on the host in extended precision (gen_twiddles.py) and compiled in
// as constants; one copy per translation unit.
#pragma once
#include <cuda_runtime.h>
#include "fft_twiddle_table.inc"

#define NSPT_FFT_MAX_LEN 512

static __constant__ double2 c_twiddle[NSPT_FFT_MAX_LEN] = {NSPT_TWIDDLE_D2};
// (cos hi, cos lo, sin hi, sin lo) as float pairs for double-float arithmetic
static __constant__ float4 c_twiddle_f4[NSPT_FFT_MAX_LEN] = {NSPT_TWIDDLE_F4};
