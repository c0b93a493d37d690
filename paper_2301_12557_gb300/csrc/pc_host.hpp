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
    // then carry the packed weights.  Binary64 weights take it through their
    // binary32 rounding hi (exponents as above) and remainder (wcorr, wlo)
    int wint = 0, wemax = 0, wemin = 0;
    int wcorr = 0;
    float *wlo = nullptr;       // cell order: remainders (GridDev::wlo), or null
    float4 *rel;
    uint16_t *cx;
    double4_32a *xw;
    int *cell_start;
    int *perm;
};

// k-d tree of Alg. 1 (tree.cu).  Nodes in heap order: slot 0 is the root,
// the children of slot h are 2h + 1 and 2h + 2; all nodes of one level hold
// floor or ceil of the same share of the points.
struct pc_tree {
    int device;
    int n;
    int weighted;
    int n_leaf;
    int depth;                  // deepest level (every node there: <= n_leaf points)
    int blevel;                 // list level: its nodes carry the traversal's lists and the
                                // origins of rel; a count splits each into balanced i-blocks
    int lmax;                   // points of the largest list node
    long long nslots;           // 2^(depth + 1) - 1
    pc::Geom g;                 // periodic and L; c = largest block extent
    double pts_lo[3], pts_hi[3];
    double r2min = 0.0;         // non-periodic: lower bound of min |x|^2
    int wint = 0, wemax = 0, wemin = 0;   // as pc_grid
    int wcorr = 0;
    float *wlo = nullptr;       // tree order: as pc_grid
    double bext = 0.0;          // largest extent (any axis) of a list node's box
    float4 *rel;                // tree order: FP32 offset from the list node's centre, .w packed weight
    double4_32a *xw;            // tree order: FP64 canonical coordinates, weight
    int *perm;                  // tree position -> input index
    int2 *vnode;                // every slot's range by the halving rule
    int2 *node;                 // {start, count} of present slots; count -1: empty slot
    double *nbox;               // lo[3], hi[3] per slot (present slots)
    signed char *naxis;         // split axis per slot, -1: leaf or empty
    double *bcen;               // list node centres, 3 per node
    int2 *brng;                 // list node ranges {start, count}
    // trees of one batched build carve their arrays from one shared device
    // block, freed with the last of them (null: arrays allocated one by one)
    struct TreeArena *arena = nullptr;
};

struct TreeArena {
    void *p = nullptr;
    int refs = 0;
};

namespace pc {

constexpr int TREE_BLOCK = 256;   // block size the automatic list level is chosen for (2 i-points)

// List-node pairs listed by the dual-tree traversal, grouped by i-node.
struct TreeLists {
    const int2 *seg = nullptr;     // {j-block, image code}
    const int *seg_off = nullptr;  // i-block -> first entry (n_i-blocks + 1)
    long long npairs = 0;
    int levels = 0;
    int nblk_i = 0;
};

// Dual-tree traversal (Alg. 3) of t1 against t2 (t1 itself for an auto
// count): node pairs whose boxes are farther apart than sqrt(r2hi), or all
// of whose pairs are closer than sqrt(r2lo), are dropped; the rest descend
// to block pairs.  The lists live in a per-device workspace valid until the
// next traversal.  Synchronises the stream once per tree level.
pc_status tree_traverse(const pc_tree *t1, const pc_tree *t2, bool is_auto, double r2hi,
                        double r2lo, cudaStream_t st, TreeLists &out);

// Balanced blocks per list node for ipt i-points per thread (NT * ipt points
// per block at most), and the pair kernel's block list of a tree count: the
// list nodes of the shard (node % shard_count == shard_index) only.
int tree_chunks(const pc_tree *t, int ipt);
cudaError_t tree_blocks(const pc_tree *t, int ipt, int shard_index, int shard_count, Block *blocks,
                        int *nblocks_dev, cudaStream_t st);

// Growable device buffer that keeps its first `keep` bytes when it grows.
struct DevVec {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes, size_t keep = 0, cudaStream_t st = nullptr) {
        if (bytes <= cap) return cudaSuccess;
        const size_t want = bytes > cap * 2 ? bytes : cap * 2;
        void *q = nullptr;
        cudaError_t e = ::pc::alloc_dev(&q, want);
        if (e != cudaSuccess) return e;
        if (keep && p) {
            e = cudaMemcpyAsync(q, p, keep, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                cudaFree(q);
                return e;
            }
        }
        if (p) cudaFree(p);
        p = q;
        cap = want;
        return cudaSuccess;
    }
};

// The concatenated lists of a batch of tree auto counts (one pair-kernel
// launch): list node k of tree t is node node0[t] + k; its blocks start at
// block0[t].
struct TreeBatch {
    std::vector<int> node0, block0;
    DevVec seg, off, rng, cen;
    long long npairs = 0;
};
pc_status tree_batch_lists(const std::vector<const pc_tree *> &ts, int ipt, double r2hi,
                           double r2lo, cudaStream_t st, TreeBatch &B);
cudaError_t tree_blocks_batch(const std::vector<const pc_tree *> &ts, const TreeBatch &B, int ipt,
                              int shard_index, int shard_count, Block *blocks, int *nblocks_dev,
                              cudaStream_t st);

// Weight checks for the integer weight path: r[0] counts weights that are
// not a non-negative normal binary32 value or zero, r[1] / r[2] the largest /
// smallest biased exponent of the non-zero ones.  Synchronises the stream.
pc_status weight_stats(const void *w, int w_is_f32, int n, cudaStream_t st, int r[4]);

// Global library lock: calls are serialised (the workspace is shared).
std::mutex &api_mutex();

// Pointer classification: true if `p` is device (or managed) memory.
bool is_device_ptr(const void *p);

// Exclusive scan of n ints into out[0..n] (out[n] = total), stream-ordered.
cudaError_t scan_exclusive(const int *in, int *out, int n, cudaStream_t st);

// Allocation-free variants: every temporary comes from the caller.
cudaError_t scan_exclusive_into(const int *in, int *out, int n, int *tot, cudaStream_t st);
// Block list: for every task t and every cell c of its i-grid in the shard
// (c % shard_count == shard_index), the cell's points split into
// ceil(count / bi) balanced blocks.  Writes the blocks (capacity must be
// >= sum over tasks of ncell + n / bi) and *nblocks.
cudaError_t make_blocks_into(const TaskDev *tasks_dev, int ntasks, int ncell, int bi,
                             int shard_index, int shard_count, Block *blocks, int *nblocks_dev,
                             int *tmp_counts, int *tmp_offsets, int *tmp_tot, cudaStream_t st);

// Forget cached count graphs that use grid g (the grid is being freed).
void forget_grid(const pc_grid *g);

// Device-side bounding box; lo/hi are host arrays (the call synchronises).
// r2min (optional) receives a lower bound of min |x|^2 over the points.
pc_status aabb_device(const double *xyz, long long n, cudaStream_t st, double *lo, double *hi,
                      double *r2min = nullptr);

}  // namespace pc
