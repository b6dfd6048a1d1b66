// Helpers the API translation unit offers to the library's other host code.
#pragma once

#include "../../include/bbs.h"

namespace bbs {
// Set the thread's last-error message and return s.
bbs_status record_error(bbs_status s, const char* msg);
// CUDA device a handle is bound to.
int handle_device(const bbs_handle* h);
}  // namespace bbs
