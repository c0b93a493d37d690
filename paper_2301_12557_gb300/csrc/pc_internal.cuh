// Internal definitions shared by the CUDA translation units of libpaircount.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "paircount.h"

namespace pc {

// ---------------------------------------------------------------------------
// launch geometry of the pair kernels
// ---------------------------------------------------------------------------
constexpr int NT = 128;        // threads per CTA (per thread group with grouped CTAs)
constexpr int TJ = 512;        // j points per shared-memory tile (FP32 path)
constexpr int TJ64 = 128;      // j points per tile (FP64 path)
constexpr int MAXSEG = 256;    // j segments per chunk of stencil rows
constexpr int MAXSEG_T = 128;  // j segments per chunk of a tree list (nodes of 129+ points;
                               // segments and their offsets fit the grid's segment space)
constexpr int ROWCHUNK = 84;   // stencil rows per chunk (<= 3 segments each)
static_assert(3 * ROWCHUNK + 1 <= MAXSEG, "a chunk's segments (and the own-cell rest) fit");
constexpr int LQ = 192;        // rescue staging slots per CTA (per thread group)
constexpr int MAX_LUT = 8192;  // LUT entries per histogram axis
// integer weight path: largest exponent range of one catalogue's weights
// (the packed significand M << range fits 32 bits), and of two catalogues'
// ranges added (a product keeps 34 bits or more: truncation below 2^-34)
constexpr int WINT_GRID_SPAN = 8;
constexpr int WINT_MAX_SPAN = 12;

enum { MODE_S = 0, MODE_SMU = 1, MODE_SIGPI = 2 };

// Remainder of a binary64 weight past its binary32 rounding hi, scaled for the
// pair kernel's correction: fl32(w - hi) 2^(142 - emax), emax the largest
// biased exponent of the catalogue's his (w - hi is exact in binary64, and
// the scaled value stays below 2^-8 in magnitude).
__device__ __forceinline__ float weight_lo(double wv, int emax) {
    const float hi = __double2float_rn(wv);
    const float lo = __double2float_rn(__dsub_rn(wv, (double)hi));
    return __double2float_rn(__dmul_rn((double)lo, ldexp(1.0, 142 - emax)));
}
enum { LOS_Z = 0, LOS_MID = 1 };

// Cell-sorted device arrays of one grid.
struct GridDev {
    const float4 *rel;       // FP32 offset from the cell centre; .w: packed integer weight
                             // (integer weight path) or 0
    const uint16_t *cx;      // x cell index per point
    const double4_32a *xw;       // FP64 canonical coordinates, .w = weight (1 if none)
    const int *cell_start;   // ncell + 1
    int n;
    // integer weight path with binary64 weights: per point the binary32
    // remainder lo = fl32(w - hi) of its weight (hi = fl32(w), the packed
    // weight) times 2^(142 - e_max), e_max the grid's largest hi exponent;
    // null when every weight is a binary32 value
    const float *wlo;
};

// One counting task: blocks of i-points of gi against the stencil of gj,
// accumulated into histogram `hist`.
struct TaskDev {
    GridDev gi, gj;
    int hist;
    int is_auto;
    double wscale;   // integer weight path: value of one unit of the product accumulators
};

// A block of consecutive i-points inside one cell.
struct Block {
    int task, cell, start, count;
};

struct Geom {
    int ng[3];
    double c[3];
    float c32[3];
    double lo[3];
    double L[3];
    double hL[3];
    int periodic;
};

// Linear lookup table over [0, T / inv_w): entries T + 2, each
// {edge (float, NaN = always rescue, +inf = no edge), k_lo (int bits)}.
struct LutDesc {
    int off;        // first entry in the concatenated table
    int T;          // cells (the table has T + 2 entries)
    float inv_w;    // cells per unit of the binned quantity
};

struct PairParams {
    const TaskDev *tasks;
    const Block *blocks;
    int *nblocks;            // device scalar
    int *work_counter;       // device scalar, zeroed per launch
    Geom g;
    const int4 *stencil;     // rows {dy, dz, xlo, xhi}
    int nrows;
    int mode, los, weighted;
    int n_a, n_b, nbins;
    float r2cut;             // FP32 candidate cut on s2
    const float2 *lut;       // concatenated LUT entries
    int lut_total;
    LutDesc la, lb;
    float eps_a, eps_b;      // rescue bands (s or sigma; pi)
    float mu_A, mu_B, mu_W;  // mu band = mu_A * (1/s) + mu_B, window mu_W
    const double *Ea;        // squared edges (device), n_a + 1
    const double *Eb;        // squared edges (device), n_b + 1
    unsigned long long *hist;    // [ntask_hist * nbins]
    double *whist;               // [ntask_hist * nbins] or null
    uint3 *queue;                // rescue queue {i, j, img | task << 5}
    unsigned long long *qcount;  // device scalar
    unsigned long long qcap;
    unsigned long long *counters;  // [0] candidates, [1] inline rescues
    int shard_index, shard_count;   // the block list holds only the cells (tree: list nodes)
                                    // whose index % shard_count == shard_index
    int groups = 1;          // FP32 kernel: independent groups of NT threads per CTA sharing
                             // one shared histogram (large histograms)
    int priv;                // 0: one histogram per CTA; 1: one per warp
    int hist_k = 1;          // lane copies of the shared histograms (power of 2, <= 32):
                             // lane l updates copy l % hist_k, stored [bin][copy]
    int smem_hist_ok;        // histogram fits in shared memory
    // evenly spaced s (and mu) edges: bins by floor instead of tables
    int lin;
    float lin_invA, lin_offA;    // t_s = s * lin_invA + lin_offA, bin = floor(t_s)
    float lin_thrA;              // not near an edge iff |frac(t_s) - 1/2| < lin_thrA
    float lin_nB;                // t_mu = mu * lin_nB
    float lin_mA, lin_cB;        // not near iff |frac(t_mu) - 1/2| < lin_cB - lin_mA / s
    // lin with e_0 = 0 and every candidate below n_a + 1 bin widths: t_s >= 0,
    // floor(t_s) <= n_a, so the s-range test is replaced by one discarded row
    // (row n_a) of the shared histogram
    int lin_norange;
    // lin with logarithmic s edges: t_s = lin_invA log2(s^2) + lin_offA, and the
    // s band grows as 1/s: not near iff |frac(t_s) - 1/2| < lin_thrA - lin_mS / s
    int lin_log;
    float lin_mS;
    // lin for (sigma, pi) bins (both axes evenly spaced from 0): t_sigma =
    // sigma lin_invA, t_pi = pi lin_invB2, not near iff |frac - 1/2| is below
    // lin_thrA and lin_thrB
    float lin_invB2, lin_thrB;
    int nbins_smem;              // bins per shared copy: nbins, plus n_b with lin_norange
    // weighted sums from exact integer products of the packed binary32 weights
    // (significand product shifted by both exponent offsets, below 2^48),
    // accumulated as three 16-bit pieces in a record of three u32 sums per bin
    // and lane copy, recombined exactly per copy and flushed as binary64 times
    // the task's wscale
    int wint;
    // integer weight path with binary64 weights (some grid carries wlo): each
    // pair's product gains the binary32 correction hi_i lo_j + lo_i hi_j,
    // rounded to the accumulators' unit, and the product is rounded instead
    // of truncated
    int wcorr;
    // integer weights with fewer than 16 lane copies (large histograms): each
    // copy reaches its product limit often, so the records are folded into
    // exact 128-bit sums per bin held for each CTA in wfold_buf (two u64 per
    // bin, low word first: gridDim x nbins x 2) instead of being flushed
    int wfold;
    unsigned long long *wfold_buf;
    int wint_k;              // lane copies of the integer weight records: hist_k
    // shared-histogram row that lanes without an in-range pair update (the
    // floor-bin kernels issue every reduction with the full warp); the flush
    // discards it like every row past nbins
    int trash_row;
    // k-d tree path (Alg. 3): each i-block (a tree node at the block level)
    // pairs with the j-blocks listed for it by the dual-tree traversal
    int tree;
    const int2 *tseg;        // {j-block, image code} per listed pair, grouped by i-block
    const int *tseg_off;     // i-block -> first entry in tseg (n_iblocks + 1)
    const int2 *tblk_j;      // j-block -> {first point, count}
    const double *tcen_i;    // i-block centres (x, y, z; binary64): the origin of rel
    const double *tcen_j;    // j-block centres
};

// ---------------------------------------------------------------------------
// error handling (host)
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
pc_status fail(pc_status s, const std::string &msg);
pc_status cuda_fail(cudaError_t e, const char *what);

// Count of kernel launches issued by the library (host side).
void note_launch(int n = 1);
long long launch_count();

// Every device (and pinned host) allocation of the library goes through these,
// which count it (pc_alloc_count).
void note_alloc();
long long alloc_count();
template <class T>
inline cudaError_t alloc_dev(T **p, size_t bytes) {
    note_alloc();
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
template <class T>
inline cudaError_t alloc_dev_async(T **p, size_t bytes, cudaStream_t st) {
    note_alloc();
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, st);
}
template <class T>
inline cudaError_t alloc_host(T **p, size_t bytes) {
    note_alloc();
    return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}

#define PC_CUDA(call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::pc::cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// launchers implemented in the kernel translation units
// ---------------------------------------------------------------------------
cudaError_t launch_pairs_f32(const PairParams &p, int ipt, int grid, size_t smem,
                             cudaStream_t st);   // p.tree selects the tree variant
cudaError_t launch_pairs_f64(const PairParams &p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_rescue(const PairParams &p, cudaStream_t st);
size_t pairs_f32_smem(const PairParams &p, int ipt);
size_t pairs_f64_smem(const PairParams &p);
int pairs_f32_ctas_per_sm(const PairParams &p, int ipt, size_t smem);
int pairs_f64_ctas_per_sm(const PairParams &p, size_t smem);

// ---------------------------------------------------------------------------
// device helpers shared by the FP32 kernel's inline rescue, the rescue
// kernel and the FP64 kernel: the exact binary64 pair definition.
// ---------------------------------------------------------------------------

// Number of k in [1, n) with v >= E[k] (E sorted); caller checked range.
__device__ __forceinline__ int f64_locate(double v, const double *E, int n) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (v >= E[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

// Largest j < n with p2 >= M[j] * s2 (the product rounded once, no FMA).
__device__ __forceinline__ int f64_locate_mu(double p2, double s2, const double *M, int n) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (p2 >= __dmul_rn(M[mid], s2)) lo = mid; else hi = mid;
    }
    return lo;
}

// Bin of the pair from binary64 separation d (already wrapped) and, for the
// midpoint line of sight, the two canonical positions.  -1: outside.
template <int MODE, int LOS>
__device__ __forceinline__ int f64_bin_from_d(double d0, double d1, double d2, const double4_32a &a,
                                              const double4_32a &b, const double *Ea, int na,
                                              const double *Eb, int nb) {
    double s2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    if (MODE == MODE_S) {
        if (!(s2 >= Ea[0] && s2 < Ea[na])) return -1;
        return f64_locate(s2, Ea, na);
    }
    double p2;
    if (LOS == LOS_Z) {
        p2 = __dmul_rn(d2, d2);
    } else {
        double l0 = __dadd_rn(a.x, b.x), l1 = __dadd_rn(a.y, b.y), l2 = __dadd_rn(a.z, b.z);
        double sl = __dadd_rn(__dadd_rn(__dmul_rn(d0, l0), __dmul_rn(d1, l1)), __dmul_rn(d2, l2));
        double ll = __dadd_rn(__dadd_rn(__dmul_rn(l0, l0), __dmul_rn(l1, l1)), __dmul_rn(l2, l2));
        p2 = (ll > 0.0) ? __ddiv_rn(__dmul_rn(sl, sl), ll) : 0.0;
    }
    if (MODE == MODE_SMU) {
        if (!(s2 >= Ea[0] && s2 < Ea[na])) return -1;
        int k = f64_locate(s2, Ea, na);
        int j = (s2 > 0.0) ? f64_locate_mu(p2, s2, Eb, nb) : 0;
        return k * nb + j;
    }
    double q2 = __dsub_rn(s2, p2);
    if (q2 < 0.0) q2 = 0.0;
    if (!(q2 >= Ea[0] && q2 < Ea[na])) return -1;
    if (!(p2 >= Eb[0] && p2 < Eb[nb])) return -1;
    return f64_locate(q2, Ea, na) * nb + f64_locate(p2, Eb, nb);
}

// Image code: (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1), s in {-1, 0, 1}: the j
// point is taken at x_j + s L.  Returns the bin under the binary64 definition
// if that image is the one the definition's wrap rule selects, -2 if it is a
// different image (that pair is counted through its own image), -1 outside.
template <int MODE, int LOS>
__device__ __forceinline__ int f64_pair_bin(const double4_32a &a, const double4_32a &b, int img,
                                            const Geom &g, const double *Ea, int na,
                                            const double *Eb, int nb) {
    double d0 = __dsub_rn(b.x, a.x);
    double d1 = __dsub_rn(b.y, a.y);
    double d2 = __dsub_rn(b.z, a.z);
    int sx = img / 9 - 1, sy = (img / 3) % 3 - 1, sz = img % 3 - 1;
    if (g.periodic) {
        int w0 = (d0 > g.hL[0]) ? -1 : ((d0 < -g.hL[0]) ? 1 : 0);
        int w1 = (d1 > g.hL[1]) ? -1 : ((d1 < -g.hL[1]) ? 1 : 0);
        int w2 = (d2 > g.hL[2]) ? -1 : ((d2 < -g.hL[2]) ? 1 : 0);
        if (w0 != sx || w1 != sy || w2 != sz) return -2;
        if (w0 < 0) d0 = __dsub_rn(d0, g.L[0]); else if (w0 > 0) d0 = __dadd_rn(d0, g.L[0]);
        if (w1 < 0) d1 = __dsub_rn(d1, g.L[1]); else if (w1 > 0) d1 = __dadd_rn(d1, g.L[1]);
        if (w2 < 0) d2 = __dsub_rn(d2, g.L[2]); else if (w2 > 0) d2 = __dadd_rn(d2, g.L[2]);
    } else if (sx != 0 || sy != 0 || sz != 0) {
        return -2;
    }
    return f64_bin_from_d<MODE, LOS>(d0, d1, d2, a, b, Ea, na, Eb, nb);
}

// floor(v * inv_w) for v >= 0 without the conversion pipe: one FFMA rounded
// toward -inf onto the 2^23 grid, then an integer subtract.  NaN/inf give a
// large index the caller clamps.
__device__ __forceinline__ int lut_index(float v, float inv_w) {
    return __float_as_int(__fmaf_rd(v, inv_w, 8388608.0f)) - 0x4B000000;
}

}  // namespace pc
