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

// Bracket the kernel launch of rfi_process_block_noalloc (whose kernel lets the launch
// after it start early): begin takes the lock under which flagging launches are
// ordered and counts the launch, end releases it.  Neither allocates; a later flagging
// launch of a context treats its stream as holding a launch with unknown buffers.
void rfi_internal_noalloc_launch_begin();
void rfi_internal_noalloc_launch_end();
