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

// Record a plain kernel launch on `stream` for the ordering of later flagging launches:
// nothing launched before it is still running once it runs; a kernel that triggers its
// successor early (triggers_early) counts as in flight with unknown buffers.
void rfi_internal_note_plain_launch(int device, void *stream, int triggers_early);
