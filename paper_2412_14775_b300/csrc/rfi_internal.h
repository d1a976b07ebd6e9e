// rfi_internal.h -- helpers shared by the library's translation units (not part of
// the public ABI).
#pragma once
#include <stddef.h>

// Record `msg` as the calling thread's last error and return `status`.
int rfi_internal_fail(int status, const char *msg);

// Check that [p, p + bytes) is device (or managed) memory of `device`, aligned to
// `align`, inside one allocation; returns RFI_OK or RFI_EINVAL (with the reason
// recorded as the last error).
int rfi_internal_check_dev(const void *p, size_t bytes, size_t align, int device,
                           const char *what);
