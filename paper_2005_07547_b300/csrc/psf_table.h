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
    unsigned* h_status;  // host-mapped pinned word written by the update (from a process-wide pool)
    unsigned host_status;           // status bits decided on the host (PSF_STATUS_SUM_RANGE)
    unsigned long long iter_vertices;  // vertices handed to inserts since the last update
    unsigned* d_status;  // its device address
    int device;
    int sms;
    int update_blocks_per_sm;  // occupancy limits of the kernels (the inserts: occ_* below)
    int query_blocks_per_sm;
    int staged_query_blocks_per_sm;  // the shared-memory staged query
    psf_launch_config launch;  // tuning knobs (psf_set_launch_config)
    // resident blocks per SM of each insert kernel variant launched so far (its grid is sized
    // from its own register use: the variants differ, and a grid above the resident limit
    // runs a partial second wave)
    mutable const void* occ_fn[16];
    mutable int occ_blocks[16];
    mutable int occ_n;
};

// Count n vertices into the table's current iteration; once the count reaches the number
// beyond which a cell's 64-bit fixed-point sum could overflow, set PSF_STATUS_SUM_RANGE.
void psf_count_iteration_vertices(psf_table* t, unsigned long long n);

// Records the CUDA error text for psf_last_cuda_error; true if e is cudaSuccess.
bool psf_cuda_ok(cudaError_t e, const char* what);
