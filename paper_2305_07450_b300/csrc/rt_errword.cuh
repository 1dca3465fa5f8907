// rt_errword.cuh -- the device error word of the library: bits set by bounded
// waits that gave up (read and cleared by rt_device_errors).  Included by the one
// translation unit that holds the kernels.
#pragma once

#include <stdint.h>

static __device__ uint32_t g_err_word;
