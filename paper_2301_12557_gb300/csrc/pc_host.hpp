// Host-side internal declarations of libpaircount.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "pc_internal.cuh"

struct pc_grid {
    int device;
    int n;
    int weighted;
    pc::Geom g;
    int ncell;
    double cell_size;           // requested cubic cell side
    double pts_lo[3], pts_hi[3];  // bounds of the (canonical) points
    double r2min = 0.0;           // non-periodic: lower bound of min |x|^2 over the points
    // integer weight path: every weight a non-negative normal binary32 value or
    // zero (wint), with biased exponents in [wemin, wemax]; the FP32 records
    // then carry the packed weights
    int wint = 0, wemax = 0, wemin = 0;
    float4 *rel;
    uint16_t *cx;
    double4_32a *xw;
    int *cell_start;
    int *perm;
};

namespace pc {

// Global library lock: calls are serialised (the workspace is shared).
std::mutex &api_mutex();

// Pointer classification: true if `p` is device (or managed) memory.
bool is_device_ptr(const void *p);

// Exclusive scan of n ints into out[0..n] (out[n] = total), stream-ordered.
cudaError_t scan_exclusive(const int *in, int *out, int n, cudaStream_t st);

// Block list: for every task t and every cell c of its i-grid, split the
// cell's points into ceil(count / bi) balanced blocks.  Writes the blocks
// (capacity must be >= sum over tasks of ncell + n / bi) and *nblocks.
cudaError_t make_blocks(const TaskDev *tasks_dev, int ntasks, int ncell, int bi, Block *blocks,
                        int *nblocks_dev, int *tmp_counts, int *tmp_offsets, cudaStream_t st);

// Allocation-free variants: every temporary comes from the caller.
cudaError_t scan_exclusive_into(const int *in, int *out, int n, int *tot, cudaStream_t st);
cudaError_t make_blocks_into(const TaskDev *tasks_dev, int ntasks, int ncell, int bi,
                             Block *blocks, int *nblocks_dev, int *tmp_counts, int *tmp_offsets,
                             int *tmp_tot, cudaStream_t st);

// Forget cached count graphs that use grid g (the grid is being freed).
void forget_grid(const pc_grid *g);

// Device-side bounding box; lo/hi are host arrays (the call synchronises).
// r2min (optional) receives a lower bound of min |x|^2 over the points.
pc_status aabb_device(const double *xyz, long long n, cudaStream_t st, double *lo, double *hi,
                      double *r2min = nullptr);

}  // namespace pc
