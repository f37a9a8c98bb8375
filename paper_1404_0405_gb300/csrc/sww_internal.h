// Read-only view of a handle for library code outside sww_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "sww.h"
#include "sww_core.cuh"

namespace sww {

struct HandleView {
    const DevLevel* jmin_level;   // the coarsest (always complete) level
    cudaStream_t stream;          // the caller's stream given to sww_create
    double radius, g, H;
};

// Fills *v; returns false for a null handle.
bool handle_view(const sww_handle* h, HandleView* v);

// Records msg as the calling thread's last error and returns code.
int set_error(int code, const char* msg);

}  // namespace sww
