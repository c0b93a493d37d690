// k-d tree on the GPU (Sect. 2.2, Alg. 1) and the dual-tree traversal
// (Sect. 3.1, Alg. 3) that lists, for every node of the list level, the
// nodes of that level (and periodic images) whose bounding boxes come within
// the largest separation.
//
// The tree is balanced (a split gives the left child floor(n / 2) points),
// so the nodes are kept in heap order: slot 0 is the root and the children
// of slot h are 2h + 1 and 2h + 2.  Every level is built by one pass of
// node statistics (sums, sums of squares and bounds per node, for the axis
// of largest variance and the minimum bounding box) and one stable radix
// sort of all points on the key (node at this level, coordinate along its
// split axis): after the sort each node's points are ordered along that
// axis and its first floor(n / 2) points are the left child.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "pc_host.hpp"

namespace pc {

// ---------------------------------------------------------------------------
// stable LSD radix sort of (u64 key, u32 value) pairs, 8 bits per pass
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;                 // threads per tile
constexpr int RS_I = 8;                   // keys per thread
constexpr int RS_TILE = RS_T * RS_I;      // keys per tile
constexpr int RS_W = RS_T / 32;           // warps per tile (each: RS_I * 32 consecutive keys)

__global__ void __launch_bounds__(RS_T) k_rs_hist(const unsigned long long *__restrict__ keys, int n,
                                                  int shift, int ntiles, int *__restrict__ cnt) {
    __shared__ int s_c[256];
    s_c[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int k = 0; k < RS_I; ++k) {
        const long long i = base + (long long)k * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&s_c[(int)((keys[i] >> shift) & 255ull)], 1);
    }
    __syncthreads();
    cnt[(size_t)threadIdx.x * ntiles + blockIdx.x] = s_c[threadIdx.x];
}

// Scatter of one tile.  Keys keep their order inside a digit: warp w holds
// the tile's keys [w * 256, w * 256 + 256) in rounds of 32, a key's place is
// the digit's global offset for this tile + the digit's count in earlier
// warps + its count earlier in its own warp (earlier rounds, lower lanes).
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const unsigned long long *__restrict__ kin,
                                                     const unsigned *__restrict__ vin,
                                                     unsigned long long *__restrict__ kout,
                                                     unsigned *__restrict__ vout, int n, int shift,
                                                     int ntiles, const int *__restrict__ off) {
    __shared__ int s_wc[RS_W][256];
    __shared__ int s_base[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < RS_W * 256; k += RS_T) (&s_wc[0][0])[k] = 0;
    s_base[threadIdx.x] = off[(size_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE + (long long)warp * (RS_I * 32);
    const unsigned below = (1u << lane) - 1u;
    unsigned long long key[RS_I];
    unsigned val[RS_I];
    int dig[RS_I], loc[RS_I];
#pragma unroll
    for (int it = 0; it < RS_I; ++it) {
        const long long i = base + it * 32 + lane;
        const bool ok = i < n;
        key[it] = ok ? kin[i] : 0ull;
        val[it] = ok ? vin[i] : 0u;
        const int d = ok ? (int)((key[it] >> shift) & 255ull) : 256 + lane;   // pads match nothing
        dig[it] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int prev = ok ? s_wc[warp][d] : 0;
        __syncwarp();
        if (ok && (peers & below) == 0u) s_wc[warp][d] = prev + __popc(peers);
        __syncwarp();
        loc[it] = prev + __popc(peers & below);
    }
    __syncthreads();
    {   // per digit: exclusive prefix of the warps' counts
        int run = 0;
        for (int w = 0; w < RS_W; ++w) {
            const int c = s_wc[w][threadIdx.x];
            s_wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_I; ++it) {
        const long long i = base + it * 32 + lane;
        if (i < n) {
            const int d = dig[it];
            const int pos = s_base[d] + s_wc[warp][d] + loc[it];
            kout[pos] = key[it];
            vout[pos] = val[it];
        }
    }
}

// Sort n pairs on key bits [0, bits); (ka, va) in and out, (kb, vb) scratch.
// cnt / off: 256 * ceil(n / RS_TILE) + 1 ints; tot: scan tile totals.
static cudaError_t radix_sort(unsigned long long *ka, unsigned *va, unsigned long long *kb,
                              unsigned *vb, int n, int bits, int *cnt, int *off, int *tot,
                              cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int ntiles = (n + RS_TILE - 1) / RS_TILE;
    unsigned long long *k0 = ka, *k1 = kb;
    unsigned *v0 = va, *v1 = vb;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        k_rs_hist<<<ntiles, RS_T, 0, st>>>(k0, n, shift, ntiles, cnt);
        note_launch();
        cudaError_t e = scan_exclusive_into(cnt, off, 256 * ntiles, tot, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<ntiles, RS_T, 0, st>>>(k0, v0, k1, v1, n, shift, ntiles, off);
        note_launch();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    if (passes & 1) {
        cudaError_t e = cudaMemcpyAsync(ka, k0, sizeof(unsigned long long) * n,
                                        cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(va, v0, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-level node statistics
// ---------------------------------------------------------------------------
__device__ __forceinline__ double canon_t(double x, double L) {
    double y = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = __dsub_rn(y, L);
    return y;
}
__device__ __forceinline__ long long okey(double v) {   // order-preserving signed key
    long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double unokey(long long k) {
    long long b = k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL);
    return __longlong_as_double(b);
}
__device__ __forceinline__ unsigned long long ukey(double v) {   // order-preserving unsigned key
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_iota(unsigned *v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (unsigned)i;
}

// canonical coordinates (periodic: folded into [0, L)) of the input points
__global__ void k_tree_canon(const double *__restrict__ xyz, int n, Geom g, double *__restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3LL * n) return;
    const int a = (int)(i % 3);
    double v = xyz[i];
    if (g.periodic) v = canon_t(v, g.L[a]);
    x[i] = v;
}

struct NodeAcc {
    double s[3], q[3];          // sums and sums of squares of (x - shift)
    long long mn[3], mx[3];     // bounds (order-preserving keys)
};

__global__ void k_acc_init(NodeAcc *acc, int m) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    NodeAcc a;
    for (int d = 0; d < 3; ++d) {
        a.s[d] = a.q[d] = 0.0;
        a.mn[d] = LLONG_MAX;
        a.mx[d] = LLONG_MIN;
    }
    acc[k] = a;
}

__device__ __forceinline__ void acc_add(NodeAcc *A, const double *s, const double *q,
                                        const long long *mn, const long long *mx) {
    for (int d = 0; d < 3; ++d) {
        atomicAdd(&A->s[d], s[d]);
        atomicAdd(&A->q[d], q[d]);
        atomicMin(&A->mn[d], mn[d]);
        atomicMax(&A->mx[d], mx[d]);
    }
}

// Statistics of the level's nodes: a warp takes 256 consecutive positions
// (nid, the node of each position at this level, never decreases along the
// positions).  A warp inside one node sums in registers and adds once; a
// warp that spans nodes reduces each round of 32 by node segments.  Sums are
// taken about `shift` (the tree's box centre); a forest of trees passes one
// centre per tree and the tree of every position (tpos), null otherwise.
__global__ void k_node_stats(const double *__restrict__ x, const unsigned *__restrict__ perm,
                             const int *__restrict__ nid, int n, double3 shift, NodeAcc *acc,
                             const double3 *__restrict__ tshift = nullptr,
                             const int *__restrict__ tpos = nullptr) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long base = gw * 256;
    if (base >= n) return;
    const long long last = min(base + 255, (long long)n - 1);
    const int n0 = nid[base], n1 = nid[last];
    if (tpos) shift = tshift[tpos[min(base + lane, last)]];   // one node: one tree
    const double sh[3] = {shift.x, shift.y, shift.z};
    if (n0 == n1) {
        double s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
        long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int it = 0; it < 8; ++it) {
            const long long i = base + it * 32 + lane;
            if (i > last) break;
            const unsigned p = perm[i];
            for (int d = 0; d < 3; ++d) {
                const double v = x[3 * (size_t)p + d];
                const double t = v - sh[d];
                s[d] += t;
                q[d] = fma(t, t, q[d]);
                mn[d] = min(mn[d], okey(v));
                mx[d] = max(mx[d], okey(v));
            }
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int d = 0; d < 3; ++d) {
                s[d] += __shfl_xor_sync(0xffffffffu, s[d], o);
                q[d] += __shfl_xor_sync(0xffffffffu, q[d], o);
                mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
                mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
            }
        if (lane == 0) acc_add(&acc[n0], s, q, mn, mx);
        return;
    }
    for (int it = 0; it < 8; ++it) {
        const long long i = base + it * 32 + lane;
        const bool ok = i <= last;
        const int node = ok ? nid[i] : -1;     // pads: one trailing segment, never added
        double s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
        long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        if (ok) {
            const unsigned p = perm[i];
            double3 shi = shift;
            if (tpos) shi = tshift[tpos[i]];
            const double shl[3] = {shi.x, shi.y, shi.z};
            for (int d = 0; d < 3; ++d) {
                const double v = x[3 * (size_t)p + d];
                const double t = v - shl[d];
                s[d] = t;
                q[d] = t * t;
                mn[d] = mx[d] = okey(v);
            }
        }
        // segmented suffix reduction: lane l ends with its segment's values
        // over [l, segment end]; segments are runs of equal node
        for (int o = 1; o < 32; o <<= 1) {
            const int on = __shfl_down_sync(0xffffffffu, node, o);
            const bool take = lane + o < 32 && on == node;
            for (int d = 0; d < 3; ++d) {
                const double ts = __shfl_down_sync(0xffffffffu, s[d], o);
                const double tq = __shfl_down_sync(0xffffffffu, q[d], o);
                const long long tn = __shfl_down_sync(0xffffffffu, mn[d], o);
                const long long tx = __shfl_down_sync(0xffffffffu, mx[d], o);
                if (take) {
                    s[d] += ts;
                    q[d] += tq;
                    mn[d] = min(mn[d], tn);
                    mx[d] = max(mx[d], tx);
                }
            }
        }
        const int up = __shfl_up_sync(0xffffffffu, node, 1);
        const bool head = ok && (lane == 0 || up != node);
        if (head) acc_add(&acc[node], s, q, mn, mx);
    }
}

// Bounds and split axis of the level's nodes (present slots only).
__global__ void k_node_finish(const NodeAcc *__restrict__ acc, int level, const int2 *__restrict__ node,
                              int n_leaf, double *__restrict__ box, signed char *__restrict__ axis) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (1 << level)) return;
    const long long h = (1LL << level) - 1 + k;
    const int2 nd = node[h];
    if (nd.y < 0) return;
    const NodeAcc A = acc[k];
    for (int d = 0; d < 3; ++d) {
        box[6 * h + d] = unokey(A.mn[d]);
        box[6 * h + 3 + d] = unokey(A.mx[d]);
    }
    int best = -1;
    if (nd.y > n_leaf) {
        // variance x count = sum (x - c)^2 - (sum (x - c))^2 / count; first maximum
        double bv = -1.0;
        for (int d = 0; d < 3; ++d) {
            const double v = A.q[d] - A.s[d] * A.s[d] / (double)nd.y;
            if (v > bv) {
                bv = v;
                best = d;
            }
        }
    }
    axis[h] = (signed char)best;
}

// ---------------------------------------------------------------------------
// the same order by chunks of whole nodes, in shared memory
// ---------------------------------------------------------------------------
// Along the positions the node ids (the keys' high bits) never decrease, so
// the stable sort of all keys only reorders the keys of each node among
// themselves.  Once every node of a level fits a chunk, one CTA per chunk of
// q whole nodes sorts its keys on (key, position) in shared memory (a bitonic
// network over the next power of two, the padding after every key) and
// writes the values back in that order: the radix sort's result, from one
// read and one write of the level's values.  With acc given it then takes
// the next level's node statistics as k_node_stats would (the children's
// ranges are the halves of each sorted node): one warp per child, its sums
// reduced in registers and stored once, with no atomics.
constexpr int CS_SMALL = 4096;    // chunk capacities (keys)
constexpr int CS_LARGE = 16384;

template <int CAP, int NTH, class R>
__global__ void __launch_bounds__(NTH) k_chunk_sort(const unsigned long long *__restrict__ keys,
                                                    unsigned *__restrict__ vals, R r,
                                                    const double *__restrict__ x, NodeAcc *acc) {
    static_assert(CAP <= 65536, "positions in a chunk are 16-bit");
    extern __shared__ __align__(16) unsigned char cs_sm[];
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(cs_sm);
    unsigned *sv = reinterpret_cast<unsigned *>(sk + CAP);
    unsigned short *si = reinterpret_cast<unsigned short *>(sv + CAP);
    const int2 rg = r.range(blockIdx.x);
    const int len = min(rg.y - rg.x, CAP);   // the host sizes chunks to CAP
    int P = 1;
    while (P < len) P <<= 1;
    for (int t = threadIdx.x; t < P; t += NTH) {
        if (t < len) {
            sk[t] = keys[rg.x + t];
            sv[t] = vals[rg.x + t];
        } else {
            sk[t] = ~0ull;
        }
        si[t] = (unsigned short)t;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += NTH) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));   // bit j clear
                const int l = i + j;
                const unsigned long long a = sk[i], b = sk[l];
                const unsigned short ia = si[i], ib = si[l];
                const bool gt = a > b || (a == b && ia > ib);
                if (gt == ((i & k) == 0)) {   // ascending where bit k of i is clear
                    sk[i] = b;
                    sk[l] = a;
                    si[i] = ib;
                    si[l] = ia;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < len; t += NTH) vals[rg.x + t] = sv[si[t]];
    if (!acc) return;
    const int lane = threadIdx.x & 31;
    const double3 sh3 = r.shift(blockIdx.x);
    const double sh[3] = {sh3.x, sh3.y, sh3.z};
    for (int c = threadIdx.x >> 5; c < 2 * r.q; c += NTH / 32) {
        const int2 nd = r.node(blockIdx.x, c >> 1);     // {first position, count}
        const int half = nd.y / 2;
        const int b0 = nd.x - rg.x + ((c & 1) ? half : 0);
        const int b1 = nd.x - rg.x + ((c & 1) ? nd.y : half);
        double s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
        long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int t = b0 + lane; t < b1; t += 32) {
            const unsigned pidx = sv[si[t]];
            for (int d = 0; d < 3; ++d) {
                const double v = x[3 * (size_t)pidx + d];
                const double tt = v - sh[d];
                s[d] += tt;
                q[d] = fma(tt, tt, q[d]);
                mn[d] = min(mn[d], okey(v));
                mx[d] = max(mx[d], okey(v));
            }
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int d = 0; d < 3; ++d) {
                s[d] += __shfl_xor_sync(0xffffffffu, s[d], o);
                q[d] += __shfl_xor_sync(0xffffffffu, q[d], o);
                mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
                mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
            }
        if (lane == 0) {
            NodeAcc A;
            for (int d = 0; d < 3; ++d) {
                A.s[d] = s[d];
                A.q[d] = q[d];
                A.mn[d] = mn[d];
                A.mx[d] = mx[d];
            }
            acc[r.child(blockIdx.x, c >> 1) + (c & 1)] = A;
        }
    }
}

// Chunk c of one tree's level: its nodes [c q, c q + q) (slots 2^d - 1 + k);
// node j of the chunk, the index of its left child one level down, and the
// centre the statistics are taken about.
struct ChunksOne {
    const int2 *vnode;
    int level, q;
    double3 centre;
    __device__ int2 range(int c) const {
        const long long h0 = (1LL << level) - 1 + (long long)c * q;
        const int2 a = vnode[h0], b = vnode[h0 + q - 1];
        return make_int2(a.x, b.x + b.y);
    }
    __device__ int2 node(int c, int j) const {
        return vnode[(1LL << level) - 1 + (long long)c * q + j];
    }
    __device__ long long child(int c, int j) const { return 2 * ((long long)c * q + j); }
    __device__ double3 shift(int) const { return centre; }
};

template <int CAP, int NTH, class R>
static cudaError_t launch_chunk_sort(const unsigned long long *keys, unsigned *vals, R r,
                                     long long chunks, const double *x, NodeAcc *acc,
                                     cudaStream_t st) {
    const size_t smem = (size_t)CAP * (sizeof(unsigned long long) + sizeof(unsigned) +
                                       sizeof(unsigned short));
    cudaError_t e = cudaFuncSetAttribute(k_chunk_sort<CAP, NTH, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chunk_sort<CAP, NTH, R><<<(unsigned)chunks, NTH, smem, st>>>(keys, vals, r, x, acc);
    note_launch();
    return cudaGetLastError();
}

// Sort level `level` by chunks when its largest node (maxsize points) fits
// one: q whole nodes a chunk, q a power of two dividing the 2^level nodes of
// each tree.  `nodes`: the level's nodes over all trees sorted.  The same
// launch leaves the statistics of level + 1 in acc (indexed as k_node_stats
// indexes them).  Returns false, launching nothing, when the nodes are too
// large.
template <class R>
static bool chunk_sort_level(const unsigned long long *keys, unsigned *vals, R r, int level,
                             long long nodes, long long maxsize, const double *x, NodeAcc *acc,
                             cudaStream_t st, cudaError_t *err) {
    const int cap = maxsize <= CS_SMALL ? CS_SMALL : (maxsize <= CS_LARGE ? CS_LARGE : 0);
    if (cap == 0) return false;
    long long q = 1;
    while (q < (1LL << level) && 2 * q * maxsize <= cap) q *= 2;
    r.level = level;
    r.q = (int)q;
    *err = cap == CS_SMALL ? launch_chunk_sort<CS_SMALL, 256>(keys, vals, r, nodes / q, x, acc, st)
                           : launch_chunk_sort<CS_LARGE, 1024>(keys, vals, r, nodes / q, x, acc, st);
    return true;
}

// Sort keys of level d: the node's index in its level on the high d bits,
// the coordinate along the node's split axis below (a node that is not
// split keeps its order: coordinate bits 0).
__global__ void k_tree_keys(const double *__restrict__ x, const unsigned *__restrict__ perm,
                            const int *__restrict__ nid, int n, int level,
                            const signed char *__restrict__ axis,
                            unsigned long long *__restrict__ keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = nid[i];
    const long long h = (1LL << level) - 1 + k;
    const int ax = axis[h];
    unsigned long long ck = 0ull;
    if (ax >= 0) ck = ukey(x[3 * (size_t)perm[i] + ax]) >> level;
    keys[i] = level ? (((unsigned long long)k << (64 - level)) | ck) : ck;
}

// Node of each position one level down (the halving rule of every slot).
__global__ void k_nid_next(const int2 *__restrict__ vnode, int n, int level, int *__restrict__ nid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = nid[i];
    const int2 v = vnode[(1LL << level) - 1 + k];
    nid[i] = 2 * k + ((i - v.x) >= v.y / 2 ? 1 : 0);
}

// List node centres (midpoints of their boxes), ranges and the largest
// extent (as an order-preserving key).
__global__ void k_block_info(const double *__restrict__ box, const int2 *__restrict__ vnode, int blevel,
                             double *__restrict__ cen, int2 *__restrict__ rng,
                             long long *__restrict__ ext_key) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (1 << blevel)) return;
    const long long h = (1LL << blevel) - 1 + b;
    double e = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double lo = box[6 * h + d], hi = box[6 * h + 3 + d];
        cen[3 * (size_t)b + d] = __dmul_rn(0.5, __dadd_rn(lo, hi));
        e = fmax(e, __dsub_rn(hi, lo));
    }
    rng[b] = vnode[h];
    atomicMax(ext_key, okey(e));
}

// Packed integer weight: the significand with its leading one shifted up by
// 8 - (emax - e) (exponents within 8 binades), as on the grid path.
__device__ __forceinline__ unsigned pack_weight_t(double wv, int emax, int span) {
    const unsigned b = __float_as_uint(__double2float_rn(wv));
    const int e = (int)((b >> 23) & 0xFF);
    if (e == 0) return 0u;
    return ((b & 0x7FFFFFu) | 0x800000u) << (span - (emax - e));
}

// Point records in tree order: FP32 offset from the list node's centre (.w the
// packed integer weight or 0), FP64 canonical coordinates and weight.
__global__ void k_tree_scatter(const double *__restrict__ x, const void *__restrict__ w, int w_is_f32,
                               int wpack_emax, int wpack_span, const unsigned *__restrict__ perm,
                               const int *__restrict__ bid, const double *__restrict__ cen, int n,
                               float4 *__restrict__ rel, double4_32a *__restrict__ xw,
                               int *__restrict__ perm_out, unsigned pbase = 0u,
                               float *__restrict__ wlo = nullptr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned p = perm[i];
    const int b = bid[i];
    double v[3];
    float r[3];
    for (int d = 0; d < 3; ++d) {
        v[d] = x[3 * (size_t)p + d];
        r[d] = __double2float_rn(__dsub_rn(v[d], cen[3 * (size_t)b + d]));
    }
    double wv = 1.0;
    if (w) wv = w_is_f32 ? (double)((const float *)w)[p] : ((const double *)w)[p];
    const unsigned wp = (w && wpack_emax > 0) ? pack_weight_t(wv, wpack_emax, wpack_span) : 0u;
    rel[i] = make_float4(r[0], r[1], r[2], __uint_as_float(wp));
    if (wlo) wlo[i] = weight_lo(wv, wpack_emax);
    xw[i] = make_double4_32a(v[0], v[1], v[2], wv);
    perm_out[i] = (int)(p - pbase);   // index into the tree's own input
}

// Levels below the root until every node holds at most cap points.
static int tree_depth(long long n, int cap) {
    int d = 0;
    long long m = n;
    while (m > cap) {
        m = (m + 1) / 2;
        ++d;
    }
    return d;
}

// ---------------------------------------------------------------------------
// dual-tree traversal (Alg. 3), one level of node pairs per launch
// ---------------------------------------------------------------------------
__device__ __forceinline__ int slot_level(int h) { return 31 - __clz(h + 1); }

// Slots for this lane's m entries in a list with counter *n: one atomic per
// warp (the lanes' counts scanned with shuffles).  Every lane of the warp
// calls it (m = 0 for none).
__device__ __forceinline__ int warp_slots(int *n, int m) {
    const int lane = threadIdx.x & 31;
    int incl = m;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(n, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - m;
}

// A node pair {a, b | image << 24}: dropped when the boxes (b shifted by
// the image) are farther apart than the largest separation or all pairs
// are closer than the smallest; listed when both are list nodes (an auto
// count leaves a node paired with itself to the pair kernel's own-node
// pass, and lists the pair from the side that balances the nodes' loads);
// otherwise split into the children pairs (a node paired with itself into
// (left, left), (left, right), (right, right)).  Splits stop at the list
// level of each tree.  The block has whole warps (256 threads): lanes past
// the list take part in the warp-wide slot allocation with nothing to add.
__global__ void __launch_bounds__(256) k_dual_level(const int2 *__restrict__ in, int n_in,
                                                    int2 *__restrict__ out, int *n_out,
                                                    int2 *__restrict__ emit, int *n_emit,
                                                    const double *__restrict__ box1,
                                                    const double *__restrict__ box2, int blev1,
                                                    int blev2, Geom g, double r2hi, double r2lo,
                                                    int is_auto) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nchild = 0, nemit = 0;
    int2 v[4];
    int2 em = make_int2(0, 0);
    if (i < n_in) {
        const int2 e = in[i];
        const int a = e.x, b = e.y & 0xFFFFFF, img = e.y >> 24;
        const int s3[3] = {img / 9 - 1, (img / 3) % 3 - 1, img % 3 - 1};
        double dmin2 = 0.0, dmax2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double sh = g.periodic ? (double)s3[d] * g.L[d] : 0.0;
            const double alo = box1[6 * (size_t)a + d], ahi = box1[6 * (size_t)a + 3 + d];
            const double blo = box2[6 * (size_t)b + d] + sh, bhi = box2[6 * (size_t)b + 3 + d] + sh;
            const double gap = fmax(0.0, fmax(blo - ahi, alo - bhi));
            const double far = fmax(bhi - alo, ahi - blo);
            dmin2 += gap * gap;
            dmax2 += far * far;
        }
        if (!(dmin2 > r2hi || dmax2 < r2lo)) {
            const bool ab = slot_level(a) >= blev1, bb = slot_level(b) >= blev2;
            const bool self = is_auto && a == b && img == 13;
            const int tag = img << 24;
            if (ab && bb) {
                if (!self) {
                    int ea = a, eb = b, ei = img;
                    if (is_auto && ((a ^ b) & 1)) {
                        ea = b;
                        eb = a;
                        ei = 26 - img;
                    }
                    em = make_int2(ea, eb | (ei << 24));
                    nemit = 1;
                }
            } else if (self) {
                v[0] = make_int2(2 * a + 1, (2 * a + 1) | tag);
                v[1] = make_int2(2 * a + 1, (2 * a + 2) | tag);
                v[2] = make_int2(2 * a + 2, (2 * a + 2) | tag);
                nchild = 3;
            } else if (!ab && !bb) {
                v[0] = make_int2(2 * a + 1, (2 * b + 1) | tag);
                v[1] = make_int2(2 * a + 1, (2 * b + 2) | tag);
                v[2] = make_int2(2 * a + 2, (2 * b + 1) | tag);
                v[3] = make_int2(2 * a + 2, (2 * b + 2) | tag);
                nchild = 4;
            } else if (ab) {
                v[0] = make_int2(a, (2 * b + 1) | tag);
                v[1] = make_int2(a, (2 * b + 2) | tag);
                nchild = 2;
            } else {
                v[0] = make_int2(2 * a + 1, b | tag);
                v[1] = make_int2(2 * a + 2, b | tag);
                nchild = 2;
            }
        }
    }
    const int ko = warp_slots(n_out, nchild);
    for (int q = 0; q < nchild; ++q) out[ko + q] = v[q];
    const int ke = warp_slots(n_emit, nemit);
    if (nemit) emit[ke] = em;
}

// Group the listed node pairs by i-node: counts, then (after a scan) the
// entries {j-node, image}; the order inside a group is arbitrary.
__global__ void k_group_count(const int2 *__restrict__ emit, int ne, int blk0, int *__restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) atomicAdd(&cnt[emit[i].x - blk0], 1);
}
__global__ void k_group_fill(const int2 *__restrict__ emit, int ne, int blk0_i, int blk0_j,
                             int *__restrict__ cursor, int2 *__restrict__ seg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int2 e = emit[i];
    const int pos = atomicAdd(&cursor[e.x - blk0_i], 1);
    seg[pos] = make_int2((e.y & 0xFFFFFF) - blk0_j, e.y >> 24);
}

// The pair kernel's blocks: every list node of the shard (nodes shard,
// shard + S, ...: nshard of them) split into k balanced chunks ("cell" = the
// list node; k is chosen so a chunk fits NT x ipt i-points).  (Batches: task
// `task`, list nodes numbered from node0, blocks written from blocks[0];
// *nblocks receives the batch's total.)
__global__ void k_tree_blocks(const int2 *__restrict__ rng, int nshard, int shard, int S, int k,
                              int task, int node0, int total, Block *__restrict__ blocks,
                              int *__restrict__ nblocks) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) *nblocks = total;
    if (b >= nshard * k) return;
    const int node = shard + S * (b / k), c = b % k;
    const int2 r = rng[node];
    const int s0 = r.x + (int)((long long)r.y * c / k), s1 = r.x + (int)((long long)r.y * (c + 1) / k);
    blocks[b] = Block{task, node0 + node, s0, s1 - s0};
}

// A tree's listed pairs appended to a batch's lists: j-nodes renumbered from
// node0, the i-node offsets shifted by the entries already there.
__global__ void k_batch_lists(const int2 *__restrict__ seg, int ne, int node0, int2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) out[i] = make_int2(seg[i].x + node0, seg[i].y);
}
__global__ void k_batch_offsets(const int *__restrict__ off, int nb, int base, int *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nb) out[i] = off[i] + base;
}

// Growable device array of the traversal workspace (reused across calls;
// the first `keep` bytes survive a growth).
struct DArr {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes, cudaStream_t st, size_t keep = 0) {
        if (bytes <= cap) return cudaSuccess;
        size_t want = std::max(bytes, cap * 2);
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

static void swap_arr(DArr &a, DArr &b) {
    std::swap(a.p, b.p);
    std::swap(a.cap, b.cap);
}

struct TraversalWs {
    DArr la, lb, emit, seg, cnt, off, cursor, tot, scal;
};

static TraversalWs &traversal_ws(int dev) {
    static std::map<int, TraversalWs> ws;
    return ws[dev];
}

pc_status tree_traverse(const pc_tree *t1, const pc_tree *t2, bool is_auto, double r2hi,
                        double r2lo, cudaStream_t st, TreeLists &out) {
    TraversalWs &W = traversal_ws(t1->device);
    const Geom &g = t1->g;
    // initial node pairs: the roots under every periodic image (an auto
    // count: the identity and the half of the images with code > 13, whose
    // mirror images would give the same pairs again)
    std::vector<int2> init;
    for (int img = 0; img < 27; ++img) {
        if (!g.periodic && img != 13) continue;
        if (is_auto && img < 13) continue;
        init.push_back(make_int2(0, img << 24));
    }
    size_t n_in = init.size();
    PC_CUDA(W.la.ensure(sizeof(int2) * n_in, st));
    PC_CUDA(W.scal.ensure(sizeof(int) * 2, st));
    PC_CUDA(cudaMemcpyAsync(W.la.p, init.data(), sizeof(int2) * n_in, cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemsetAsync(W.scal.p, 0, sizeof(int) * 2, st));
    int *d_nout = (int *)W.scal.p, *d_nemit = d_nout + 1;
    long long n_emit = 0;
    int levels = 0;
    while (n_in > 0) {
        const size_t out_cap = 4 * n_in;
        if (out_cap > (size_t)INT_MAX || (size_t)n_emit + n_in > (size_t)INT_MAX)
            return fail(PC_EOVERFLOW, "tree traversal: too many node pairs");
        PC_CUDA(W.lb.ensure(sizeof(int2) * out_cap, st));
        PC_CUDA(W.emit.ensure(sizeof(int2) * ((size_t)n_emit + n_in), st, sizeof(int2) * n_emit));
        PC_CUDA(cudaMemsetAsync(d_nout, 0, sizeof(int), st));
        k_dual_level<<<(unsigned)((n_in + 255) / 256), 256, 0, st>>>(
            (const int2 *)W.la.p, (int)n_in, (int2 *)W.lb.p, d_nout, (int2 *)W.emit.p, d_nemit,
            t1->nbox, t2->nbox, t1->blevel, t2->blevel, g, r2hi, r2lo, is_auto ? 1 : 0);
        note_launch();
        PC_CUDA(cudaGetLastError());
        int h[2];
        PC_CUDA(cudaMemcpyAsync(h, W.scal.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        PC_CUDA(cudaStreamSynchronize(st));
        n_in = (size_t)h[0];
        n_emit = h[1];
        swap_arr(W.la, W.lb);
        ++levels;
    }
    // group by i-node
    const int nbi = 1 << t1->blevel;
    const int blk0_i = nbi - 1, blk0_j = (1 << t2->blevel) - 1;
    const size_t ne = (size_t)n_emit;
    PC_CUDA(W.seg.ensure(sizeof(int2) * std::max<size_t>(ne, 1), st));
    PC_CUDA(W.cnt.ensure(sizeof(int) * (nbi + 1), st));
    PC_CUDA(W.off.ensure(sizeof(int) * (nbi + 1), st));
    PC_CUDA(W.cursor.ensure(sizeof(int) * (nbi + 1), st));
    PC_CUDA(W.tot.ensure(sizeof(int) * ((nbi + 1) / 4096 + 2), st));
    PC_CUDA(cudaMemsetAsync(W.cnt.p, 0, sizeof(int) * (nbi + 1), st));
    if (ne > 0) {
        k_group_count<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>((const int2 *)W.emit.p, (int)ne,
                                                                     blk0_i, (int *)W.cnt.p);
        note_launch();
    }
    PC_CUDA(scan_exclusive_into((const int *)W.cnt.p, (int *)W.off.p, nbi, (int *)W.tot.p, st));
    PC_CUDA(cudaMemcpyAsync(W.cursor.p, W.off.p, sizeof(int) * (nbi + 1), cudaMemcpyDeviceToDevice, st));
    if (ne > 0) {
        k_group_fill<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
            (const int2 *)W.emit.p, (int)ne, blk0_i, blk0_j, (int *)W.cursor.p, (int2 *)W.seg.p);
        note_launch();
    }
    PC_CUDA(cudaGetLastError());
    out.seg = (const int2 *)W.seg.p;
    out.seg_off = (const int *)W.off.p;
    out.npairs = (long long)ne;
    out.levels = levels;
    out.nblk_i = nbi;
    return PC_OK;
}

int tree_chunks(const pc_tree *t, int ipt) {
    const int cap = NT * ipt;
    return std::max(1, (t->lmax + cap - 1) / cap);
}

// List nodes of a shard among nl: shard, shard + S, ... below nl.
static int shard_nodes(int nl, int shard, int S) { return nl > shard ? (nl - shard + S - 1) / S : 0; }

cudaError_t tree_blocks(const pc_tree *t, int ipt, int shard_index, int shard_count, Block *blocks,
                        int *nblocks_dev, cudaStream_t st) {
    if (shard_count < 1) shard_count = 1, shard_index = 0;
    const int nl = 1 << t->blevel;
    const int k = tree_chunks(t, ipt);
    const int ns = shard_nodes(nl, shard_index, shard_count);
    const int nb = ns * k;
    k_tree_blocks<<<std::max(1, (nb + 255) / 256), 256, 0, st>>>(t->brng, ns, shard_index,
                                                                 shard_count, k, 0, 0, nb, blocks,
                                                                 nblocks_dev);
    note_launch();
    return cudaGetLastError();
}

pc_status tree_batch_lists(const std::vector<const pc_tree *> &ts, int ipt, double r2hi, double r2lo,
                           cudaStream_t st, TreeBatch &B) {
    const int m = (int)ts.size();
    B.node0.assign(m + 1, 0);
    B.block0.assign(m + 1, 0);
    for (int k = 0; k < m; ++k) {
        const int nl = 1 << ts[k]->blevel;
        B.node0[k + 1] = B.node0[k] + nl;
        B.block0[k + 1] = B.block0[k] + nl * tree_chunks(ts[k], ipt);
    }
    const int nn = B.node0[m];
    PC_CUDA(B.off.ensure(sizeof(int) * ((size_t)nn + 1)));
    PC_CUDA(B.rng.ensure(sizeof(int2) * (size_t)nn));
    PC_CUDA(B.cen.ensure(sizeof(double) * 3 * (size_t)nn));
    long long nseg = 0;
    for (int k = 0; k < m; ++k) {
        TreeLists TL;
        pc_status s = tree_traverse(ts[k], ts[k], true, r2hi, r2lo, st, TL);
        if (s != PC_OK) return s;
        if (nseg + TL.npairs > (long long)INT_MAX)
            return fail(PC_EOVERFLOW, "tree batch: too many listed node pairs");
        // the traversal workspace is reused by the next tree: append now
        PC_CUDA(B.seg.ensure(sizeof(int2) * (size_t)std::max<long long>(nseg + TL.npairs, 1),
                             sizeof(int2) * (size_t)nseg, st));
        const int nl = 1 << ts[k]->blevel;
        if (TL.npairs > 0) {
            k_batch_lists<<<(unsigned)((TL.npairs + 255) / 256), 256, 0, st>>>(
                TL.seg, (int)TL.npairs, B.node0[k], (int2 *)B.seg.p + nseg);
            note_launch();
        }
        k_batch_offsets<<<(nl + 1 + 255) / 256, 256, 0, st>>>(TL.seg_off, nl, (int)nseg,
                                                              (int *)B.off.p + B.node0[k]);
        note_launch();
        PC_CUDA(cudaMemcpyAsync((int2 *)B.rng.p + B.node0[k], ts[k]->brng, sizeof(int2) * nl,
                                cudaMemcpyDeviceToDevice, st));
        PC_CUDA(cudaMemcpyAsync((double *)B.cen.p + 3 * (size_t)B.node0[k], ts[k]->bcen,
                                sizeof(double) * 3 * nl, cudaMemcpyDeviceToDevice, st));
        PC_CUDA(cudaGetLastError());
        // the next traversal overwrites the lists: finish the copies first
        PC_CUDA(cudaStreamSynchronize(st));
        nseg += TL.npairs;
    }
    B.npairs = nseg;
    return PC_OK;
}

cudaError_t tree_blocks_batch(const std::vector<const pc_tree *> &ts, const TreeBatch &B, int ipt,
                              int shard_index, int shard_count, Block *blocks, int *nblocks_dev,
                              cudaStream_t st) {
    (void)B;
    if (shard_count < 1) shard_count = 1, shard_index = 0;
    const int m = (int)ts.size();
    // blocks of every tree's shard, back to back
    std::vector<int> b0(m + 1, 0);
    for (int k = 0; k < m; ++k)
        b0[k + 1] = b0[k] + shard_nodes(1 << ts[k]->blevel, shard_index, shard_count) *
                                tree_chunks(ts[k], ipt);
    for (int k = 0; k < m; ++k) {
        const int ns = shard_nodes(1 << ts[k]->blevel, shard_index, shard_count);
        const int kc = tree_chunks(ts[k], ipt);
        k_tree_blocks<<<std::max(1, (ns * kc + 255) / 256), 256, 0, st>>>(
            ts[k]->brng, ns, shard_index, shard_count, kc, k, B.node0[k], b0[m], blocks + b0[k],
            nblocks_dev);
        note_launch();
    }
    return cudaGetLastError();
}

// Points of the largest node of level d (the halving rule).
static long long level_largest(long long n, int d) {
    long long m = n;
    for (int k = 0; k < d; ++k) m = (m + 1) / 2;
    return m;
}

// List level: the level whose nodes carry the traversal's lists and the
// origins of the FP32 offsets.  cap > 0: the first level whose nodes hold at
// most cap points; cap = 0: among the levels whose largest node holds 129 to
// 2048 points, the one whose nodes split into TREE_BLOCK-point blocks with
// the fewest idle i-slots (the deepest on a tie; a catalogue of at most
// TREE_BLOCK points: the root).
static int list_level(long long n, int cap) {
    int best = tree_depth(n, cap > 0 ? cap : TREE_BLOCK);
    if (cap == 0) {
        double bf = -1.0;
        for (int d = 0; d <= 40; ++d) {
            const long long m = level_largest(n, d);
            if (m > 2048) continue;
            if (m <= TREE_BLOCK / 2 && d > 0) break;
            const long long k = (m + TREE_BLOCK - 1) / TREE_BLOCK;
            const double fill = (double)n / (double)(1LL << d) / (double)(k * TREE_BLOCK);
            if (fill >= bf - 1e-12) {
                bf = fill;
                best = d;
            }
            if (m <= TREE_BLOCK) break;
        }
    }
    return best;
}

}  // namespace pc

// ---------------------------------------------------------------------------
// public: tree build / free / info / export
// ---------------------------------------------------------------------------
using namespace pc;

static void tree_release(pc_tree *t) {
    if (!t) return;
    cudaFree(t->wlo);   // never carved from a batch's block
    if (t->arena) {   // arrays carved from a batch's shared block
        if (--t->arena->refs == 0) {
            cudaFree(t->arena->p);
            delete t->arena;
        }
        delete t;
        return;
    }
    cudaFree(t->rel);
    cudaFree(t->xw);
    cudaFree(t->perm);
    cudaFree(t->vnode);
    cudaFree(t->node);
    cudaFree(t->nbox);
    cudaFree(t->naxis);
    cudaFree(t->bcen);
    cudaFree(t->brng);
    delete t;
}

extern "C" void pc_free_tree(pc_tree *t) {
    std::lock_guard<std::mutex> lk(api_mutex());
    tree_release(t);
}

extern "C" pc_status pc_tree_info(const pc_tree *t, long long *n, int *depth, int *list_level,
                                  long long *slots) {
    if (!t) return fail(PC_EINVAL, "pc_tree_info: null tree");
    if (n) *n = t->n;
    if (depth) *depth = t->depth;
    if (list_level) *list_level = t->blevel;
    if (slots) *slots = t->nslots;
    return PC_OK;
}

extern "C" pc_status pc_tree_export(const pc_tree *t, long long *start, long long *count, int *axis,
                                    double *box, long long *ord) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!t) return fail(PC_EINVAL, "pc_tree_export: null tree");
    const size_t ns = (size_t)t->nslots;
    if (start || count) {
        std::vector<int2> nd(ns);
        PC_CUDA(cudaMemcpy(nd.data(), t->node, sizeof(int2) * ns, cudaMemcpyDeviceToHost));
        for (size_t h = 0; h < ns; ++h) {
            if (start) start[h] = nd[h].y >= 0 ? nd[h].x : 0;
            if (count) count[h] = nd[h].y;
        }
    }
    if (axis) {
        std::vector<signed char> ax(ns);
        PC_CUDA(cudaMemcpy(ax.data(), t->naxis, ns, cudaMemcpyDeviceToHost));
        for (size_t h = 0; h < ns; ++h) axis[h] = ax[h];
    }
    if (box) PC_CUDA(cudaMemcpy(box, t->nbox, sizeof(double) * 6 * ns, cudaMemcpyDeviceToHost));
    if (ord && t->n > 0) {
        std::vector<int> pm(t->n);
        PC_CUDA(cudaMemcpy(pm.data(), t->perm, sizeof(int) * t->n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < t->n; ++i) ord[i] = pm[i];
    }
    return PC_OK;
}

extern "C" pc_status pc_build_tree(const double *xyz, const void *w, int w_is_f32, long long n,
                                   const pc_box *box, int n_leaf, int list_cap, void *stream,
                                   pc_tree **out) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!out) return fail(PC_EINVAL, "pc_build_tree: out is NULL");
    *out = nullptr;
    if (!box) return fail(PC_EINVAL, "pc_build_tree: box is NULL");
    if (n < 1) return fail(PC_EINVAL, "pc_build_tree: a tree needs at least one point");
    if (!xyz) return fail(PC_EINVAL, "pc_build_tree: xyz is NULL");
    if (n >= (1LL << 31) - 1) return fail(PC_EOVERFLOW, "pc_build_tree: n must be below 2^31");
    if (n_leaf < 1 || n_leaf > 128) return fail(PC_EINVAL, "pc_build_tree: n_leaf must lie in [1, 128]");
    if (list_cap != 0 && (list_cap < TREE_BLOCK || list_cap > 65536 || (list_cap & (list_cap - 1))))
        return fail(PC_EINVAL, "pc_build_tree: list_cap must be 0 or a power of two in [256, 65536]");
    const int depth = tree_depth(n, n_leaf);
    const int blevel = std::min(list_level(n, list_cap), depth);
    if (depth > 27) return fail(PC_EOVERFLOW, "pc_build_tree: more than 2^28 tree slots");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));

    pc_tree *t = new pc_tree();
    memset(static_cast<void *>(t), 0, sizeof(*t));
    t->device = dev;
    t->n = (int)n;
    t->weighted = (w != nullptr);
    t->n_leaf = n_leaf;
    t->depth = depth;
    t->blevel = blevel;
    t->lmax = (int)level_largest(n, blevel);
    t->nslots = (2LL << depth) - 1;
    Geom &G = t->g;
    G.periodic = box->periodic ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        if (G.periodic) {
            if (!(box->L[a] > 0.0) || !isfinite(box->L[a])) {
                delete t;
                return fail(PC_EINVAL, "pc_build_tree: periodic box needs L > 0 on every axis");
            }
            G.L[a] = box->L[a];
            G.hL[a] = 0.5 * box->L[a];
        }
        G.ng[a] = 1;
    }

    // temporaries
    std::vector<void *> tmp;
    auto talloc = [&](void **p, size_t bytes) {
        cudaError_t e = ::pc::alloc_dev_async(p, std::max<size_t>(bytes, 16), st);
        if (e == cudaSuccess) tmp.push_back(*p);
        return e;
    };
    auto cleanup = [&]() {
        for (void *p : tmp) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    };
    auto bail = [&](pc_status s) {
        cleanup();
        tree_release(t);
        return s;
    };
    const double *dxyz = xyz;
    const void *dw = w;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(xyz)) {
        void *q = nullptr;
        e = talloc(&q, sizeof(double) * 3 * n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        dxyz = (const double *)q;
    }
    const size_t wbytes = (size_t)n * (w_is_f32 ? sizeof(float) : sizeof(double));
    if (e == cudaSuccess && w && !is_device_ptr(w)) {
        void *q = nullptr;
        e = talloc(&q, wbytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q, w, wbytes, cudaMemcpyHostToDevice, st);
        dw = q;
    }
    double *x = nullptr;
    if (e == cudaSuccess) e = talloc((void **)&x, sizeof(double) * 3 * n);
    if (e == cudaSuccess) {
        k_tree_canon<<<(unsigned)((3 * n + 255) / 256), 256, 0, st>>>(dxyz, (int)n, G, x);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "pc_build_tree: inputs"));

    // bounds of the canonical points and, non-periodic, the smallest radius
    double plo[3], phi[3];
    {
        pc_status s = aabb_device(x, n, st, plo, phi, G.periodic ? nullptr : &t->r2min);
        if (s != PC_OK) return bail(s);
        for (int a = 0; a < 3; ++a)
            if (!isfinite(plo[a]) || !isfinite(phi[a]))
                return bail(fail(PC_EINVAL, "pc_build_tree: non-finite coordinates"));
        for (int a = 0; a < 3; ++a) {
            t->pts_lo[a] = G.periodic ? 0.0 : plo[a];
            t->pts_hi[a] = G.periodic ? G.L[a] : phi[a];
            G.lo[a] = t->pts_lo[a];
        }
    }
    // weights usable by the integer weight path (binary64 weights with their
    // remainders, as on the grid path)
    if (dw) {
        int r[4];
        pc_status s = weight_stats(dw, w_is_f32, (int)n, st, r);
        if (s != PC_OK) return bail(s);
        if (r[0] == 0 && (r[1] < 0 || r[1] - r[2] <= WINT_GRID_SPAN)) {
            t->wint = 1;
            t->wemax = r[1] >= 0 ? r[1] : 1;
            t->wemin = r[1] >= 0 ? r[2] : 1;
            t->wcorr = r[3] > 0 ? 1 : 0;
            if (t->wcorr) {
                cudaError_t ea = ::pc::alloc_dev(&t->wlo, sizeof(float) * (size_t)n);
                if (ea != cudaSuccess) {
                    cudaGetLastError();
                    return bail(fail(PC_ENOMEM, "pc_build_tree: device allocation failed"));
                }
            }
        }
    }

    // slot ranges by the halving rule (also below leaves: "virtual" ranges
    // keep those points in place during the sorts); present slots: the root
    // and the children of split nodes
    const size_t ns = (size_t)t->nslots;
    std::vector<int2> vnode(ns), node(ns);
    vnode[0] = make_int2(0, (int)n);
    node[0] = vnode[0];
    for (size_t h = 0; 2 * h + 2 < ns; ++h) {
        const int2 v = vnode[h];
        vnode[2 * h + 1] = make_int2(v.x, v.y / 2);
        vnode[2 * h + 2] = make_int2(v.x + v.y / 2, v.y - v.y / 2);
        const bool split = node[h].y > n_leaf;
        node[2 * h + 1] = split ? vnode[2 * h + 1] : make_int2(0, -1);
        node[2 * h + 2] = split ? vnode[2 * h + 2] : make_int2(0, -1);
    }
    e = ::pc::alloc_dev(&t->vnode, sizeof(int2) * ns);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->node, sizeof(int2) * ns);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->nbox, sizeof(double) * 6 * ns);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->naxis, ns);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->rel, sizeof(float4) * n);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->xw, sizeof(double4_32a) * n);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->perm, sizeof(int) * n);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->bcen, sizeof(double) * 3 * ((size_t)1 << blevel));
    if (e == cudaSuccess) e = ::pc::alloc_dev(&t->brng, sizeof(int2) * ((size_t)1 << blevel));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PC_ENOMEM, "pc_build_tree: device allocation failed"));
    }
    e = cudaMemcpyAsync(t->vnode, vnode.data(), sizeof(int2) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->node, node.data(), sizeof(int2) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->naxis, 0xFF, ns, st);   // -1: leaf or empty
    if (e == cudaSuccess) e = cudaMemsetAsync(t->nbox, 0, sizeof(double) * 6 * ns, st);

    // level loop
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    unsigned long long *ka = nullptr, *kb = nullptr;
    unsigned *va = nullptr, *vb = nullptr;
    int *nid = nullptr, *bid = nullptr, *cnt = nullptr, *off = nullptr, *tot = nullptr;
    NodeAcc *acc = nullptr;
    long long *ext = nullptr;
    const size_t ncnt = (size_t)256 * ntiles + 1;
    if (e == cudaSuccess) e = talloc((void **)&ka, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = talloc((void **)&kb, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = talloc((void **)&va, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = talloc((void **)&vb, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = talloc((void **)&nid, sizeof(int) * n);
    if (e == cudaSuccess) e = talloc((void **)&bid, sizeof(int) * n);
    if (e == cudaSuccess) e = talloc((void **)&cnt, sizeof(int) * ncnt);
    if (e == cudaSuccess) e = talloc((void **)&off, sizeof(int) * ncnt);
    if (e == cudaSuccess) e = talloc((void **)&tot, sizeof(int) * (ncnt / 4096 + 2));
    if (e == cudaSuccess) e = talloc((void **)&acc, sizeof(NodeAcc) * ((size_t)1 << depth));
    if (e == cudaSuccess) e = talloc((void **)&ext, sizeof(long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PC_ENOMEM, "pc_build_tree: device allocation failed"));
    }
    if (e == cudaSuccess) {
        k_iota<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(va, (int)n);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(nid, 0, sizeof(int) * n, st);
    const double3 shift = make_double3(0.5 * (t->pts_lo[0] + t->pts_hi[0]),
                                       0.5 * (t->pts_lo[1] + t->pts_hi[1]),
                                       0.5 * (t->pts_lo[2] + t->pts_hi[2]));
    const unsigned gpos = (unsigned)((n + 255) / 256);
    bool stats_done = false;   // the previous level's chunk sort left this level's statistics
    for (int d = 0; e == cudaSuccess && d <= depth; ++d) {
        const int m = 1 << d;
        if (!stats_done) {
            k_acc_init<<<(m + 255) / 256, 256, 0, st>>>(acc, m);
            note_launch();
            const long long warps = (n + 255) / 256;
            k_node_stats<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(x, va, nid, (int)n,
                                                                                 shift, acc);
            note_launch();
        }
        k_node_finish<<<(m + 255) / 256, 256, 0, st>>>(acc, d, t->node, n_leaf, t->nbox, t->naxis);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess && d == blevel)
            e = cudaMemcpyAsync(bid, nid, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess || d == depth) break;
        k_tree_keys<<<gpos, 256, 0, st>>>(x, va, nid, (int)n, d, t->naxis, ka);
        note_launch();
        ChunksOne co{t->vnode, d, 1, shift};
        stats_done = chunk_sort_level(ka, va, co, d, 1LL << d, (n + (1LL << d) - 1) >> d, x, acc,
                                      st, &e);
        if (!stats_done) e = radix_sort(ka, va, kb, vb, (int)n, 64, cnt, off, tot, st);
        if (e == cudaSuccess) {
            k_nid_next<<<gpos, 256, 0, st>>>(t->vnode, (int)n, d, nid);
            note_launch();
            e = cudaGetLastError();
        }
    }
    // list nodes and point records
    const int nblk = 1 << blevel;
    long long ext_init = LLONG_MIN, ext_key = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ext, &ext_init, sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_block_info<<<(nblk + 255) / 256, 256, 0, st>>>(t->nbox, t->vnode, blevel, t->bcen, t->brng, ext);
        note_launch();
        k_tree_scatter<<<gpos, 256, 0, st>>>(x, dw, w_is_f32, t->wint ? t->wemax : 0,
                                             WINT_GRID_SPAN, va, bid, t->bcen,
                                             (int)n, t->rel, t->xw, t->perm, 0u, t->wlo);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ext_key, ext, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pc_build_tree"));
    {
        long long b = ext_key >= 0 ? ext_key : (ext_key ^ 0x7FFFFFFFFFFFFFFFLL);
        double ex;
        memcpy(&ex, &b, sizeof(ex));
        t->bext = ex;
    }
    for (int a = 0; a < 3; ++a) {
        G.c[a] = std::max(t->bext, 1e-300);
        G.c32[a] = (float)G.c[a];
    }
    cleanup();
    *out = t;
    return PC_OK;
}

// ---------------------------------------------------------------------------
// batched build: the k-d trees of many catalogues in one level loop
// ---------------------------------------------------------------------------
// The catalogues' points are laid end to end, the deepest tree first, so the
// trees still being split at level d are a prefix of the arrays.  At level d
// tree r (its rank in that order) owns the global node ids r 2^d .. r 2^d +
// 2^d - 1; id g's children are 2g and 2g + 1, so one set of node
// statistics, one key pass and one radix sort per level serve every tree,
// and each tree ends with the same node ranges, boxes and split axes as its
// own build (statistics summed in another order may break an exact variance
// tie the other way: a different but equally valid median split).
namespace pc {

struct FTree {
    int2 *vnode, *node;
    double *nbox;
    signed char *naxis;
    long long pos;     // first position of the tree's points
    int n, n_leaf, depth, blevel;
};

// Chunk c of a forest's level: global nodes [c q, c q + q), all of one tree
// (q divides the 2^d nodes of each); node j, its left child's global id one
// level down, and the tree's centre.
struct ChunksForest {
    const FTree *ft;
    int level, q;
    const double3 *centres;
    __device__ int2 range(int c) const {
        const long long g0 = (long long)c * q;
        const FTree &T = ft[g0 >> level];
        const long long h0 = (1LL << level) - 1 + (g0 & ((1LL << level) - 1));
        const int2 a = T.vnode[h0], b = T.vnode[h0 + q - 1];
        return make_int2((int)(T.pos + a.x), (int)(T.pos + b.x + b.y));
    }
    __device__ int2 node(int c, int j) const {
        const long long g = (long long)c * q + j;
        const FTree &T = ft[g >> level];
        const int2 v = T.vnode[(1LL << level) - 1 + (g & ((1LL << level) - 1))];
        return make_int2((int)(T.pos + v.x), v.y);
    }
    __device__ long long child(int c, int j) const { return 2 * ((long long)c * q + j); }
    __device__ double3 shift(int c) const { return centres[((long long)c * q) >> level]; }
};

__global__ void k_fnode_finish(const NodeAcc *__restrict__ acc, int level, int ntrees,
                               const FTree *__restrict__ ft) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ((long long)ntrees << level)) return;
    const FTree &T = ft[g >> level];
    const long long h = (1LL << level) - 1 + (g & ((1LL << level) - 1));
    const int2 nd = T.node[h];
    if (nd.y < 0) return;
    const NodeAcc A = acc[g];
    for (int d = 0; d < 3; ++d) {
        T.nbox[6 * h + d] = unokey(A.mn[d]);
        T.nbox[6 * h + 3 + d] = unokey(A.mx[d]);
    }
    int best = -1;
    if (nd.y > T.n_leaf) {
        double bv = -1.0;
        for (int d = 0; d < 3; ++d) {
            const double v = A.q[d] - A.s[d] * A.s[d] / (double)nd.y;
            if (v > bv) {
                bv = v;
                best = d;
            }
        }
    }
    T.naxis[h] = (signed char)best;
}

// Sort keys of level d over the trees being split: the global node id on
// the high d + rbits bits (rbits: enough for the number of trees), the
// coordinate along the node's split axis below.
__global__ void k_ftree_keys(const double *__restrict__ x, const unsigned *__restrict__ perm,
                             const int *__restrict__ nid, long long n, int level, int rbits,
                             const FTree *__restrict__ ft, unsigned long long *__restrict__ keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = nid[i];
    const FTree &T = ft[g >> level];
    const long long h = (1LL << level) - 1 + (g & ((1 << level) - 1));
    const int ax = T.naxis[h];
    const int hb = level + rbits;
    unsigned long long ck = 0ull;
    if (ax >= 0) ck = ukey(x[3 * (size_t)perm[i] + ax]) >> hb;
    keys[i] = hb ? (((unsigned long long)g << (64 - hb)) | ck) : ck;
}

// Global node of each position one level down.
__global__ void k_fnid_next(const FTree *__restrict__ ft, long long n, int level, int *__restrict__ nid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = nid[i];
    const FTree &T = ft[g >> level];
    const int2 v = T.vnode[(1LL << level) - 1 + (g & ((1 << level) - 1))];
    nid[i] = 2 * g + ((int)(i - T.pos - v.x) >= v.y / 2 ? 1 : 0);
}

// List node (local to its tree) of the positions of trees whose list level is d.
__global__ void k_fbid(const int *__restrict__ nid, const int *__restrict__ tpos, long long n, int level,
                       const FTree *__restrict__ ft, int *__restrict__ bid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ft[tpos[i]].blevel == level) bid[i] = nid[i] & ((1 << level) - 1);
}

// Slot ranges of level d by the halving rule, for the trees with a level d
// (global node g = r 2^d + k): level 0 is the root {0, n}; a slot's children
// are present while it holds more than n_leaf points.
__global__ void k_fslots(int level, int ntrees, const FTree *__restrict__ ft) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ((long long)ntrees << level)) return;
    const FTree &T = ft[g >> level];
    if (level == 0) {
        T.vnode[0] = make_int2(0, T.n);
        T.node[0] = T.vnode[0];
        return;
    }
    const long long k = g & ((1LL << level) - 1);
    const long long h = (1LL << level) - 1 + k;
    const long long hp = (1LL << (level - 1)) - 1 + (k >> 1);
    const int2 v = T.vnode[hp];
    const int2 c = (k & 1) ? make_int2(v.x + v.y / 2, v.y - v.y / 2) : make_int2(v.x, v.y / 2);
    T.vnode[h] = c;
    T.node[h] = T.node[hp].y > T.n_leaf ? c : make_int2(0, -1);
}

// Canonical coordinates in place (periodic: folded into [0, L)).
__global__ void k_fcanon(double *x, long long n3, Geom g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3 || !g.periodic) return;
    x[i] = canon_t(x[i], g.L[i % 3]);
}

__global__ void k_fill_int(int *__restrict__ a, long long n0, long long n1, int v) {
    const long long i = n0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) a[i] = v;
}

}  // namespace pc

extern "C" pc_status pc_build_tree_batch(const double *const *xyz, const void *const *w, int w_is_f32,
                                         const long long *n, int m, const pc_box *box, int n_leaf,
                                         int list_cap, void *stream, pc_tree **out) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!out || !xyz || !n || !box || m < 1)
        return fail(PC_EINVAL, "pc_build_tree_batch: bad arguments");
    for (int k = 0; k < m; ++k) out[k] = nullptr;
    if (m > (1 << 16)) return fail(PC_EOVERFLOW, "pc_build_tree_batch: more than 65536 catalogues");
    if (n_leaf < 1 || n_leaf > 128)
        return fail(PC_EINVAL, "pc_build_tree_batch: n_leaf must lie in [1, 128]");
    if (list_cap != 0 && (list_cap < TREE_BLOCK || list_cap > 65536 || (list_cap & (list_cap - 1))))
        return fail(PC_EINVAL, "pc_build_tree_batch: list_cap must be 0 or a power of two in [256, 65536]");
    const bool weighted = w && w[0];
    long long N = 0;
    for (int k = 0; k < m; ++k) {
        if (!xyz[k] || n[k] < 1) return fail(PC_EINVAL, "pc_build_tree_batch: every catalogue needs points");
        if (weighted != (w && w[k] != nullptr))
            return fail(PC_EINVAL, "pc_build_tree_batch: weights for all catalogues or none");
        N += n[k];
    }
    if (N >= (1LL << 31) - 1) return fail(PC_EOVERFLOW, "pc_build_tree_batch: more than 2^31 points");
    Geom G0{};
    G0.periodic = box->periodic ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        if (G0.periodic) {
            if (!(box->L[a] > 0.0) || !isfinite(box->L[a]))
                return fail(PC_EINVAL, "pc_build_tree_batch: periodic box needs L > 0 on every axis");
            G0.L[a] = box->L[a];
            G0.hL[a] = 0.5 * box->L[a];
        }
        G0.ng[a] = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));

    // the deepest tree first; positions end to end in that order
    std::vector<int> depth(m), blev(m), ord(m);
    int dmax = 0;
    for (int k = 0; k < m; ++k) {
        depth[k] = tree_depth(n[k], n_leaf);
        blev[k] = std::min(list_level(n[k], list_cap), depth[k]);
        if (depth[k] > 27) return fail(PC_EOVERFLOW, "pc_build_tree_batch: more than 2^28 tree slots");
        dmax = std::max(dmax, depth[k]);
        ord[k] = k;
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return depth[a] > depth[b]; });
    std::vector<long long> pos(m + 1, 0), nmax(m + 1, 0);   // nmax[a]: largest of the first a trees
    for (int r = 0; r < m; ++r) {
        pos[r + 1] = pos[r] + n[ord[r]];
        nmax[r + 1] = std::max(nmax[r], n[ord[r]]);
    }

    std::vector<pc_tree *> trees(m, nullptr);
    std::vector<void *> tmp;
    auto talloc = [&](void **p, size_t bytes) {
        cudaError_t e = ::pc::alloc_dev_async(p, std::max<size_t>(bytes, 16), st);
        if (e == cudaSuccess) tmp.push_back(*p);
        return e;
    };
    auto bail = [&](pc_status s) {
        for (void *p : tmp) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
        for (pc_tree *t : trees) tree_release(t);
        return s;
    };

    // the points end to end (canonical), the weights likewise, the tree of
    // every position
    double *x = nullptr;
    void *wall = nullptr;
    int *tpos = nullptr;
    const size_t wsz = w_is_f32 ? sizeof(float) : sizeof(double);
    cudaError_t e = talloc((void **)&x, sizeof(double) * 3 * (size_t)N);
    if (e == cudaSuccess && weighted) e = talloc(&wall, wsz * (size_t)N);
    if (e == cudaSuccess) e = talloc((void **)&tpos, sizeof(int) * (size_t)N);
    for (int r = 0; e == cudaSuccess && r < m; ++r) {
        const int k = ord[r];
        e = cudaMemcpyAsync(x + 3 * pos[r], xyz[k], sizeof(double) * 3 * n[k],
                            is_device_ptr(xyz[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && weighted)
            e = cudaMemcpyAsync((char *)wall + wsz * pos[r], w[k], wsz * n[k],
                                is_device_ptr(w[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            k_fill_int<<<(unsigned)((n[k] + 255) / 256), 256, 0, st>>>(tpos, pos[r], pos[r + 1], r);
            note_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_fcanon<<<(unsigned)((3 * N + 255) / 256), 256, 0, st>>>(x, 3 * N, G0);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "pc_build_tree_batch: inputs"));

    // every tree: bounds and weights; its arrays carved from one device block
    // shared by the batch (freed with the last tree)
    std::vector<FTree> ft(m);
    std::vector<double3> shifts(m);
    if (G0.periodic) {   // one bounds pass over the forest: finite coordinates
        double plo[3], phi[3];
        pc_status s = aabb_device(x, N, st, plo, phi, nullptr);
        if (s != PC_OK) return bail(s);
        for (int a = 0; a < 3; ++a)
            if (!isfinite(plo[a]) || !isfinite(phi[a]))
                return bail(fail(PC_EINVAL, "pc_build_tree_batch: non-finite coordinates"));
    }
    auto carve = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
    size_t total = 0;
    for (int r = 0; r < m; ++r) {
        const int k = ord[r];
        const size_t ns = ((size_t)2 << depth[k]) - 1, nb = (size_t)1 << blev[k], nk = (size_t)n[k];
        total += carve(sizeof(int2) * ns) * 2 + carve(sizeof(double) * 6 * ns) + carve(ns) +
                 carve(sizeof(float4) * nk) + carve(sizeof(double4_32a) * nk) + carve(sizeof(int) * nk) +
                 carve(sizeof(double) * 3 * nb) + carve(sizeof(int2) * nb);
    }
    TreeArena *arena = new TreeArena();
    e = ::pc::alloc_dev(&arena->p, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete arena;
        return bail(fail(PC_ENOMEM, "pc_build_tree_batch: device allocation failed"));
    }
    char *cur = (char *)arena->p;
    auto take = [&](size_t bytes) {
        char *p = cur;
        cur += carve(bytes);
        return (void *)p;
    };
    for (int r = 0; r < m; ++r) {
        const int k = ord[r];
        pc_tree *t = new pc_tree();
        memset(static_cast<void *>(t), 0, sizeof(*t));
        trees[r] = t;
        t->arena = arena;
        arena->refs += 1;
        t->device = dev;
        t->n = (int)n[k];
        t->weighted = weighted ? 1 : 0;
        t->n_leaf = n_leaf;
        t->depth = depth[k];
        t->blevel = blev[k];
        t->lmax = (int)level_largest(n[k], blev[k]);
        t->nslots = (2LL << depth[k]) - 1;
        t->g = G0;
        const size_t ns = (size_t)t->nslots, nb = (size_t)1 << blev[k];
        t->vnode = (int2 *)take(sizeof(int2) * ns);
        t->node = (int2 *)take(sizeof(int2) * ns);
        t->nbox = (double *)take(sizeof(double) * 6 * ns);
        t->naxis = (signed char *)take(ns);
        t->rel = (float4 *)take(sizeof(float4) * n[k]);
        t->xw = (double4_32a *)take(sizeof(double4_32a) * n[k]);
        t->perm = (int *)take(sizeof(int) * n[k]);
        t->bcen = (double *)take(sizeof(double) * 3 * nb);
        t->brng = (int2 *)take(sizeof(int2) * nb);
        const double *xs = x + 3 * pos[r];
        pc_status s = PC_OK;
        if (G0.periodic) {
            for (int a = 0; a < 3; ++a) { t->pts_lo[a] = 0.0; t->pts_hi[a] = G0.L[a]; }
        } else {
            double plo[3], phi[3];
            s = aabb_device(xs, n[k], st, plo, phi, &t->r2min);
            if (s != PC_OK) return bail(s);
            for (int a = 0; a < 3; ++a) {
                if (!isfinite(plo[a]) || !isfinite(phi[a]))
                    return bail(fail(PC_EINVAL, "pc_build_tree_batch: non-finite coordinates"));
                t->pts_lo[a] = plo[a];
                t->pts_hi[a] = phi[a];
            }
        }
        for (int a = 0; a < 3; ++a) t->g.lo[a] = t->pts_lo[a];
        shifts[r] = make_double3(0.5 * (t->pts_lo[0] + t->pts_hi[0]), 0.5 * (t->pts_lo[1] + t->pts_hi[1]),
                                 0.5 * (t->pts_lo[2] + t->pts_hi[2]));
        if (weighted) {
            int res[4];
            s = weight_stats((const char *)wall + wsz * pos[r], w_is_f32, (int)n[k], st, res);
            if (s != PC_OK) return bail(s);
            if (res[0] == 0 && (res[1] < 0 || res[1] - res[2] <= WINT_GRID_SPAN)) {
                t->wint = 1;
                t->wemax = res[1] >= 0 ? res[1] : 1;
                t->wemin = res[1] >= 0 ? res[2] : 1;
                t->wcorr = res[3] > 0 ? 1 : 0;
                if (t->wcorr) {   // its own allocation, outside the shared block
                    cudaError_t ea = ::pc::alloc_dev(&t->wlo, sizeof(float) * (size_t)n[k]);
                    if (ea != cudaSuccess) {
                        cudaGetLastError();
                        return bail(fail(PC_ENOMEM, "pc_build_tree_batch: device allocation failed"));
                    }
                }
            }
        }
        e = cudaMemsetAsync(t->naxis, 0xFF, ns, st);   // -1: leaf or empty
        if (e == cudaSuccess) e = cudaMemsetAsync(t->nbox, 0, sizeof(double) * 6 * ns, st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "pc_build_tree_batch: tree arrays"));
        ft[r] = FTree{t->vnode, t->node, t->nbox, t->naxis, pos[r], (int)n[k], n_leaf, depth[k], blev[k]};
    }

    // trees still being split at each level (a prefix of the rank order)
    std::vector<int> active(dmax + 2, 0);
    for (int d = 0; d <= dmax + 1; ++d)
        while (active[d] < m && depth[ord[active[d]]] >= d) ++active[d];
    long long acc_n = 1;
    for (int d = 0; d <= dmax; ++d) acc_n = std::max(acc_n, (long long)active[d] << d);

    FTree *dft = nullptr;
    double3 *dshift = nullptr;
    unsigned long long *ka = nullptr, *kb = nullptr;
    unsigned *va = nullptr, *vb = nullptr;
    int *nid = nullptr, *bid = nullptr, *cnt = nullptr, *off = nullptr, *tot = nullptr;
    NodeAcc *acc = nullptr;
    long long *ext = nullptr;
    const int ntiles = (int)((N + RS_TILE - 1) / RS_TILE);
    const size_t ncnt = (size_t)256 * ntiles + 1;
    e = talloc((void **)&dft, sizeof(FTree) * m);
    if (e == cudaSuccess) e = talloc((void **)&dshift, sizeof(double3) * m);
    if (e == cudaSuccess) e = talloc((void **)&ka, sizeof(unsigned long long) * N);
    if (e == cudaSuccess) e = talloc((void **)&kb, sizeof(unsigned long long) * N);
    if (e == cudaSuccess) e = talloc((void **)&va, sizeof(unsigned) * N);
    if (e == cudaSuccess) e = talloc((void **)&vb, sizeof(unsigned) * N);
    if (e == cudaSuccess) e = talloc((void **)&nid, sizeof(int) * N);
    if (e == cudaSuccess) e = talloc((void **)&bid, sizeof(int) * N);
    if (e == cudaSuccess) e = talloc((void **)&cnt, sizeof(int) * ncnt);
    if (e == cudaSuccess) e = talloc((void **)&off, sizeof(int) * ncnt);
    if (e == cudaSuccess) e = talloc((void **)&tot, sizeof(int) * (ncnt / 4096 + 2));
    if (e == cudaSuccess) e = talloc((void **)&acc, sizeof(NodeAcc) * acc_n);
    if (e == cudaSuccess) e = talloc((void **)&ext, sizeof(long long) * m);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PC_ENOMEM, "pc_build_tree_batch: device allocation failed"));
    }
    e = cudaMemcpyAsync(dft, ft.data(), sizeof(FTree) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dshift, shifts.data(), sizeof(double3) * m, cudaMemcpyHostToDevice, st);
    const unsigned gall = (unsigned)((N + 255) / 256);
    if (e == cudaSuccess) {
        k_iota<<<gall, 256, 0, st>>>(va, (int)N);
        note_launch();
        e = cudaMemcpyAsync(nid, tpos, sizeof(int) * N, cudaMemcpyDeviceToDevice, st);   // level 0: id = rank
    }
    int rbits = 0;
    bool stats_done = false;   // the previous level's chunk sort left this level's statistics
    for (int d = 0; e == cudaSuccess && d <= dmax; ++d) {
        const int A = active[d];                  // trees with a level d
        const long long nA = pos[A];              // their positions
        const long long gm = (long long)A << d;   // their level-d nodes
        k_fslots<<<(unsigned)((gm + 255) / 256), 256, 0, st>>>(d, A, dft);
        note_launch();
        if (!stats_done) {
            k_acc_init<<<(unsigned)((gm + 255) / 256), 256, 0, st>>>(acc, (int)gm);
            note_launch();
            const long long warps = (nA + 255) / 256;
            k_node_stats<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
                x, va, nid, (int)nA, make_double3(0, 0, 0), acc, dshift, tpos);
            note_launch();
        }
        k_fnode_finish<<<(unsigned)((gm + 255) / 256), 256, 0, st>>>(acc, d, A, dft);
        note_launch();
        k_fbid<<<(unsigned)((nA + 255) / 256), 256, 0, st>>>(nid, tpos, nA, d, dft, bid);
        note_launch();
        e = cudaGetLastError();
        const int A2 = active[d + 1];             // trees split below level d
        const long long nS = pos[A2];
        if (e != cudaSuccess || A2 == 0) break;
        rbits = 0;
        while ((1 << rbits) < A2) ++rbits;
        k_ftree_keys<<<(unsigned)((nS + 255) / 256), 256, 0, st>>>(x, va, nid, nS, d, rbits, dft, ka);
        note_launch();
        ChunksForest cf{dft, d, 1, dshift};
        stats_done = chunk_sort_level(ka, va, cf, d, (long long)A2 << d,
                                      (nmax[A2] + (1LL << d) - 1) >> d, x, acc, st, &e);
        if (!stats_done) e = radix_sort(ka, va, kb, vb, (int)nS, 64, cnt, off, tot, st);
        if (e == cudaSuccess) {
            k_fnid_next<<<(unsigned)((nS + 255) / 256), 256, 0, st>>>(dft, nS, d, nid);
            note_launch();
            e = cudaGetLastError();
        }
    }
    // list nodes and point records, tree by tree
    std::vector<long long> ext_key(m, 0);
    {
        std::vector<long long> init(m, LLONG_MIN);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ext, init.data(), sizeof(long long) * m, cudaMemcpyHostToDevice, st);
        for (int r = 0; e == cudaSuccess && r < m; ++r) {
            pc_tree *t = trees[r];
            const int nblk = 1 << t->blevel;
            k_block_info<<<(nblk + 255) / 256, 256, 0, st>>>(t->nbox, t->vnode, t->blevel, t->bcen, t->brng,
                                                              ext + r);
            note_launch();
            k_tree_scatter<<<(unsigned)((t->n + 255) / 256), 256, 0, st>>>(
                x, wall, w_is_f32, t->wint ? t->wemax : 0, WINT_GRID_SPAN, va + pos[r],
                bid + pos[r], t->bcen, t->n, t->rel, t->xw, t->perm, (unsigned)pos[r], t->wlo);
            note_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ext_key.data(), ext, sizeof(long long) * m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "pc_build_tree_batch"));
    for (int r = 0; r < m; ++r) {
        pc_tree *t = trees[r];
        long long b = ext_key[r] >= 0 ? ext_key[r] : (ext_key[r] ^ 0x7FFFFFFFFFFFFFFFLL);
        double ex;
        memcpy(&ex, &b, sizeof(ex));
        t->bext = ex;
        for (int a = 0; a < 3; ++a) {
            t->g.c[a] = std::max(t->bext, 1e-300);
            t->g.c32[a] = (float)t->g.c[a];
        }
    }
    for (void *p : tmp) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    for (int r = 0; r < m; ++r) out[ord[r]] = trees[r];
    return PC_OK;
}
