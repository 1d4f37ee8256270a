// psf_table.h -- host-side table header shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "psf.h"
#include "psf_device.cuh"

struct psf_table {
    psf_config cfg;
    psf::TableView view;
    void* mem;
    size_t bytes;
    unsigned* h_status;  // host-mapped pinned word written by the update
    int device;
    int sms;
    int insert_blocks_per_sm;  // occupancy limits of the kernels
    int update_blocks_per_sm;
    int query_blocks_per_sm;
    int staged_blocks_per_sm;  // the shared-memory staged insert and query
    int staged_query_blocks_per_sm;
    psf_launch_config launch;  // tuning knobs (psf_set_launch_config)
};

// Records the CUDA error text for psf_last_cuda_error; true if e is cudaSuccess.
bool psf_cuda_ok(cudaError_t e, const char* what);
