// Pair-separation histogram kernels (templates; instantiated per binning
// mode in pairs_*.cu).
//
// Work decomposition (grid traversal of Sect. 2.1 with the half-shell
// duplicate removal of Sect. 3.1): a persistent CTA (or each of its thread
// groups) repeatedly takes a block of up to NT * RI consecutive points of one
// cell (the i-points, kept in registers) and streams every candidate j-point
// of the neighbouring cells through shared memory.  Neighbours are visited row
// by row: for a stencil row (dy, dz) the cells (ax + xlo .. ax + xhi, ay + dy,
// az + dz) are contiguous in the cell-sorted arrays, so each row is one index
// range (split at most in three by periodic wrapping).  Periodic images are
// handled by shifting whole cells (Sect. 3.1), never by testing each pair.
// Runs of 32 staged j-points are skipped per warp when their bounding box is
// out of reach of the warp's i-points.
//
// FP32 path: the j-point is staged as its offset from the i-cell centre,
// rel_j + delta * c, so a pair costs three subtractions and three
// multiply-adds.  The squared separation selects candidates; in-range pairs
// are binned by floors of scaled values (evenly spaced or logarithmic s,
// evenly spaced mu, sigma and pi; Sect. 3.2.2) or through lookup tables for
// other edges (Sect. 3.2.3), each table entry holding the single bin edge
// near that table cell.  A pair whose value lies within the proven FP32 error
// band of an edge is re-evaluated with the exact binary64 definition (queued
// for the rescue kernel), so the integer counts equal the binary64 definition
// exactly.
#pragma once

#include "pc_internal.cuh"

namespace pc {

constexpr unsigned long long FLUSH_LIMIT = 1ull << 30;
// integer weight path: products (each < 2^48) per lane copy between flushes;
// each of its three u32 piece sums then adds less than 2^16 pieces of 16
// bits, and the copy's recombined sum stays below 2^64.  With binary64
// remainders (W == 3) a product is below 2^49, its top piece below 2^17,
// and half as many products fit.
constexpr unsigned long long WINT_LIMIT = 1ull << 16;

struct SmemLayout {
    size_t lut, ea, eb, hist, whist, seg, tile, meta, tw, q, total;
    size_t gstride;   // per-group area [seg, q end): group g's copy is g * gstride further
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// FP32 path (f64 = false) and FP64 path (f64 = true) share one layout.
__host__ __device__ inline SmemLayout smem_layout(const PairParams &p, bool f64) {
    SmemLayout L;
    size_t o = 0;
    L.lut = o;
    o = align_up(o + (size_t)p.lut_total * sizeof(float2), 16);
    // squared edges: the FP64 kernel's binning (the FP32 kernel's rescue
    // reads them from global memory)
    L.ea = o;
    if (f64) o = align_up(o + (size_t)(p.n_a + 1) * sizeof(double), 16);
    L.eb = o;
    if (f64) o = align_up(o + (size_t)(p.n_b + 1) * sizeof(double), 16);
    int copies = (p.priv ? NT / 32 : 1) * p.hist_k;
    L.hist = o;
    if (p.smem_hist_ok) o = align_up(o + (size_t)p.nbins_smem * copies * sizeof(int), 16);
    L.whist = o;
    if (p.smem_hist_ok && p.weighted) {
        if (p.wint && !f64)   // records of three u32 sums of 16-bit product pieces
            o = align_up(o + (size_t)3 * p.nbins_smem * p.wint_k * sizeof(unsigned), 16);
        else
            o = align_up(o + (size_t)p.nbins_smem * p.hist_k * sizeof(double), 16);
    }
    L.seg = o;
    o = align_up(o + (size_t)(p.tree && !f64 ? MAXSEG_T : MAXSEG) * sizeof(int4), 16);
    int tj = f64 ? TJ64 : TJ;
    L.tile = o;
    o = align_up(o + (size_t)2 * tj * (f64 ? sizeof(double4_32a) : 3 * sizeof(float)), 16);
    L.meta = o;
    if (f64) o = align_up(o + (size_t)2 * tj * sizeof(int2), 16);
    else if (p.tree) o = align_up(o + (size_t)MAXSEG_T * sizeof(float4), 16);   // segment offsets
    // staged j weights: binary64, or the packed 4-byte integer weights (and,
    // with binary64 remainders, the 4-byte remainders after them)
    L.tw = o;
    if (p.weighted && !f64)
        o = align_up(o + (size_t)2 * tj * (p.wint ? (p.wcorr ? 2 : 1) * sizeof(unsigned) : sizeof(double)), 16);
    L.q = o;
    o = align_up(o + (size_t)LQ * sizeof(uint3), 16);
    L.gstride = o - L.seg;
    L.total = L.seg + (size_t)(f64 ? 1 : p.groups) * L.gstride;
    return L;
}

// ---------------------------------------------------------------------------
// thread groups: a CTA of G groups of NT threads; each group works on its own
// blocks and synchronises only with itself (named barrier 1 + group)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int gtid() { return (int)(threadIdx.x % NT); }

template <int G>
__device__ __forceinline__ void gsync() {
    if (G == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / NT)), "r"(NT) : "memory");
    }
}

template <int G>
__device__ __forceinline__ bool gsync_or(bool v) {
    if (G == 1) return __syncthreads_or(v) != 0;
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "r"(1 + (int)(threadIdx.x / NT)), "r"(NT)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------
// per-CTA state shared by both precisions
// ---------------------------------------------------------------------------
struct CtaShared {
    int blk;
    int nseg;
    int total;
    int qn;
    unsigned long long pruned;   // candidate pairs decided by group bounds
};

// Axis-aligned box of a group of points in the i-cell's FP32 frame.
struct GBox {
    float4 lo, hi;
};
constexpr int JG = 32;           // j-points per bounding-box group
static_assert(TJ % JG == 0 && TJ / JG <= 32, "group masks are one 32-bit ballot");
static_assert(NT % JG == 0 && (JG == 16 || JG == 32), "each warp stages whole groups");

// Order-preserving map of binary32 onto int32 (its own inverse): a < b as
// floats iff fkey(a) < fkey(b) as signed integers.
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }
__device__ __forceinline__ float warp_minf(float v) {
    return fkey_inv(__reduce_min_sync(0xffffffffu, fkey(v)));
}
__device__ __forceinline__ float warp_maxf(float v) {
    return fkey_inv(__reduce_max_sync(0xffffffffu, fkey(v)));
}

// Box of the JG consecutive lanes that hold one staged j-group (lanes
// without a point pass valid = false); every lane gets its group's box.
__device__ __forceinline__ GBox lane_group_box(float x, float y, float z, bool valid) {
    float lx = valid ? x : INFINITY, ly = valid ? y : INFINITY, lz = valid ? z : INFINITY;
    float hx = valid ? x : -INFINITY, hy = valid ? y : -INFINITY, hz = valid ? z : -INFINITY;
    if (JG == 32) {
        lx = warp_minf(lx); ly = warp_minf(ly); lz = warp_minf(lz);
        hx = warp_maxf(hx); hy = warp_maxf(hy); hz = warp_maxf(hz);
    } else {
#pragma unroll
        for (int o = JG / 2; o > 0; o >>= 1) {   // stays inside each half-warp
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
    }
    return GBox{make_float4(lx, ly, lz, 0.f), make_float4(hx, hy, hz, 0.f)};
}

// Groups of the staged tile that may hold a pair in range of this warp's
// i-points.  Bit g is clear only if, for every i of the warp and every j of
// group g, the kernel's own FP32 value fl(fl(dz dz + fl(dy dy + fl(dx dx))))
// would be >= r2cut: |fl(x_j - x_i)| >= fl(gap) per axis because rounding is
// monotone, and the same operations on the gaps give a lower bound of s2.
// So the skipped pairs are exactly pairs the kernel would reject one by one.
// Group g of tile `tile` is the chunk's group g * fstride + tile; the last
// group of the chunk may hold fewer than JG points (of `total`).
__device__ __forceinline__ unsigned group_mask(const GBox *gb, const GBox &ib, int ngroups,
                                               int tile, int fstride, int total, int ni,
                                               float r2cut, unsigned long long *pruned) {
    const int lane = threadIdx.x & 31;
    bool keep = false;
    if (lane < ngroups) {
        const GBox g = gb[lane];
        const float gx = fmaxf(fmaxf(g.lo.x - ib.hi.x, ib.lo.x - g.hi.x), 0.f);
        const float gy = fmaxf(fmaxf(g.lo.y - ib.hi.y, ib.lo.y - g.hi.y), 0.f);
        const float gz = fmaxf(fmaxf(g.lo.z - ib.hi.z, ib.lo.z - g.hi.z), 0.f);
        keep = fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < r2cut;
        if (!keep && ni > 0) {
            const int first = (lane * fstride + tile) * JG;
            atomicAdd(pruned, (unsigned long long)min(JG, total - first) * (unsigned)ni);
        }
    }
    return __ballot_sync(0xffffffffu, keep);
}

// Exclusive prefix over the segment lengths held in seg[k].y (in place);
// returns the total.  All NT threads call it.
template <int G = 1>
__device__ __forceinline__ int seg_scan(int4 *seg, int nseg, int *s_tmp) {
    // each thread owns a contiguous run of ceil(nseg / NT) segments
    const int tid = gtid();
    const int per = (nseg + NT - 1) / NT;
    int b0 = tid * per, b1 = min(b0 + per, nseg);
    int local = 0;
    for (int k = b0; k < b1; ++k) local += seg[k].y;
    // block-wide exclusive scan of `local` (NT = 128: 4 warps)
    int lane = tid & 31, warp = tid >> 5;
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_tmp[warp] = v;
    gsync<G>();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_tmp[w];
    int total = s_tmp[0] + s_tmp[1] + s_tmp[2] + s_tmp[3];
    int run = wbase + v - local;
    for (int k = b0; k < b1; ++k) {
        int len = seg[k].y;
        seg[k].y = run;
        run += len;
    }
    gsync<G>();
    return total;
}

// Segment holding flat position f: largest k with seg[k].y <= f.
__device__ __forceinline__ int seg_find(const int4 *seg, int nseg, int f) {
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (seg[mid].y <= f) lo = mid; else hi = mid;
    }
    return lo;
}

// Build the j-segments of stencil rows [r0, r1) for the i-cell (ax, ay, az).
// seg = {first point, length, dy | dz << 16, image code}.
__device__ __forceinline__ void build_segments(const PairParams &p, const GridDev &gj, int ax,
                                               int ay, int az, int r0, int r1, int4 *seg,
                                               int *s_nseg) {
    const int nx = p.g.ng[0], ny = p.g.ng[1], nz = p.g.ng[2];
    for (int row = r0 + gtid(); row < r1; row += NT) {
        int4 st = p.stencil[row];
        int dy = st.x, dz = st.y;
        int y = ay + dy, z = az + dz, wy = 0, wz = 0;
        if (y < 0) { if (!p.g.periodic) continue; y += ny; wy = -1; }
        else if (y >= ny) { if (!p.g.periodic) continue; y -= ny; wy = 1; }
        if (z < 0) { if (!p.g.periodic) continue; z += nz; wz = -1; }
        else if (z >= nz) { if (!p.g.periodic) continue; z -= nz; wz = 1; }
        const int rowbase = (z * ny + y) * nx;
        const int x0 = ax + st.z, x1 = ax + st.w;
        int pc0[3], pc1[3], pw[3], np = 0;
        if (p.g.periodic) {
            if (x0 < 0) { pc0[np] = x0 + nx; pc1[np] = min(x1, -1) + nx; pw[np++] = -1; }
            int m0 = max(x0, 0), m1 = min(x1, nx - 1);
            if (m0 <= m1) { pc0[np] = m0; pc1[np] = m1; pw[np++] = 0; }
            if (x1 >= nx) { pc0[np] = max(x0, nx) - nx; pc1[np] = x1 - nx; pw[np++] = 1; }
        } else {
            int m0 = max(x0, 0), m1 = min(x1, nx - 1);
            if (m0 <= m1) { pc0[np] = m0; pc1[np] = m1; pw[np++] = 0; }
        }
        const int meta = (dy & 0xFFFF) | (dz << 16);
        for (int q = 0; q < np; ++q) {
            int a0 = gj.cell_start[rowbase + pc0[q]];
            int a1 = gj.cell_start[rowbase + pc1[q] + 1];
            if (a1 > a0) {
                int slot = atomicAdd(s_nseg, 1);
                seg[slot] = make_int4(a0, a1 - a0, meta, (pw[q] + 1) * 9 + (wy + 1) * 3 + (wz + 1));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// rescue helpers
// ---------------------------------------------------------------------------
template <int MODE, int LOS, bool COUNT = true>
__device__ __noinline__ void inline_rescue(const PairParams &p, uint3 e) {
    const int task = (int)(e.z >> 5), img = (int)(e.z & 31);
    const TaskDev &T = p.tasks[task];
    double4_32a a = T.gi.xw[e.x];
    double4_32a b = T.gj.xw[e.y];
    int bin = f64_pair_bin<MODE, LOS>(a, b, img, p.g, p.Ea, p.n_a, p.Eb, p.n_b);
    if (bin >= 0) {
        size_t h = (size_t)T.hist * p.nbins + bin;
        atomicAdd(&p.hist[h], 1ull);
        if (p.weighted) atomicAdd(&p.whist[h], __dmul_rn(a.w, b.w));
    }
    if (COUNT) atomicAdd(&p.counters[1], 1ull);
}

template <int MODE, int LOS>
__device__ __forceinline__ void push_rescue(const PairParams &p, uint3 *s_q, int *s_qn, uint3 e) {
    int slot = atomicAdd(s_qn, 1);
    if (slot < LQ) {
        s_q[slot] = e;
        return;
    }
    unsigned long long g = atomicAdd(p.qcount, 1ull);
    if (g < p.qcap) p.queue[g] = e;
    else inline_rescue<MODE, LOS>(p, e);
}

// Drain the CTA's staged rescue entries to the global queue.  All threads
// call it, after a barrier that follows their last push, so every thread
// reads the same count.
template <int MODE, int LOS, int G = 1>
__device__ __forceinline__ void drain_rescue(const PairParams &p, uint3 *s_q, CtaShared &cs,
                                             unsigned long long *s_base) {
    int n = min(cs.qn, LQ);
    if (n == 0) return;
    const int tid = gtid();
    if (tid == 0) *s_base = atomicAdd(p.qcount, (unsigned long long)n);
    gsync<G>();
    unsigned long long base = *s_base;
    for (int k = tid; k < n; k += NT) {
        unsigned long long g = base + k;
        if (g < p.qcap) p.queue[g] = s_q[k];
        else inline_rescue<MODE, LOS, false>(p, s_q[k]);
    }
    // entries past the queue were evaluated here: one counter update per drain
    if (tid == 0 && base + n > p.qcap)
        atomicAdd(&p.counters[1], base + n - max(base, p.qcap));
    gsync<G>();
    if (tid == 0) cs.qn = 0;
    gsync<G>();
}

// Read a shared counter and clear it.  With several thread groups sharing
// the histogram another group may be adding to it meanwhile: exchange.
template <int G>
__device__ __forceinline__ int take_i32(int *a) {
    if (G == 1) {
        const int v = *a;
        *a = 0;
        return v;
    }
    return atomicExch(a, 0);
}
template <int G>
__device__ __forceinline__ unsigned long long take_u64(unsigned long long *a) {
    if (G == 1) {
        const unsigned long long v = *a;
        *a = 0ull;
        return v;
    }
    return atomicExch(a, 0ull);
}

// Fold mode (integer weights, one thread group): the exact sum of bin b's
// lane-copy records as a 128-bit value (lo, hi), the records cleared; each
// copy's sum is below 2^64.
__device__ __forceinline__ void fold_bin(const PairParams &p, unsigned *wp, int b,
                                         unsigned long long &lo, unsigned long long &hi) {
    lo = 0ull;
    hi = 0ull;
    for (int k = 0; k < p.wint_k; ++k) {
        unsigned *r = wp + ((size_t)b * p.wint_k + k) * 3;
        const unsigned long long t = (unsigned long long)r[0] + ((unsigned long long)r[1] << 16) +
                                     ((unsigned long long)r[2] << 32);
        r[0] = r[1] = r[2] = 0u;
        lo += t;
        hi += lo < t ? 1ull : 0ull;
    }
}

// Fold mode: every bin's records into this CTA's 128-bit sums in wfold_buf
// (bin b is always handled by thread b mod NT, here and in flush_hist, so a
// CTA's sums need no atomics); the counts stay in their copies.
__device__ __forceinline__ void fold_records(const PairParams &p, double *s_whist) {
    __syncthreads();
    unsigned *wp = reinterpret_cast<unsigned *>(s_whist);
    for (int b = threadIdx.x; b < p.nbins_smem; b += NT) {
        unsigned long long lo, hi;
        fold_bin(p, wp, b, lo, hi);
        if (b < p.nbins && (lo | hi)) {
            unsigned long long *f = p.wfold_buf + ((size_t)blockIdx.x * p.nbins + b) * 2;
            const unsigned long long l1 = f[0] + lo;
            f[1] += hi + (l1 < lo ? 1ull : 0ull);
            f[0] = l1;
        }
    }
    __syncthreads();
}

// Add the shared histogram(s) into histogram `h` and clear them (all threads
// of the calling group; with G > 1 each group flushes whatever has been
// added so far, which the exchanges take exactly once).
template <int G = 1>
__device__ __forceinline__ void flush_hist(const PairParams &p, int *s_hist, double *s_whist,
                                           int h, double wscale = 0.0) {
    gsync<G>();
    if (p.smem_hist_ok && h >= 0) {
        // layout [warp copy][bin][lane copy]; bins past nbins form the
        // discarded row of lin_norange and are only cleared
        const int copies = p.priv ? NT / 32 : 1, K = p.hist_k, nbs = p.nbins_smem;
        unsigned long long *u = reinterpret_cast<unsigned long long *>(s_whist);
        unsigned *wp = reinterpret_cast<unsigned *>(s_whist);   // integer weight records
        const int WK = p.wint_k;
        for (int b = gtid(); b < nbs; b += NT) {
            long long v = 0;
            for (int c = 0; c < copies; ++c)
                for (int k = 0; k < K; ++k) v += take_i32<G>(&s_hist[(c * nbs + b) * K + k]);
            if (b >= p.nbins) {   // discarded rows (and the row of lanes without a pair)
                if (p.weighted && p.wint) {
                    for (int q = 0; q < 3 * WK; ++q) take_i32<G>((int *)&wp[(size_t)b * 3 * WK + q]);
                } else if (p.weighted) {
                    for (int k = 0; k < K; ++k) take_u64<G>(&u[b * K + k]);
                }
                continue;
            }
            if (v) atomicAdd(&p.hist[(size_t)h * p.nbins + b], (unsigned long long)v);
            if (p.weighted) {
                double w = 0.0;
                if (p.wint && p.wfold) {
                    // this CTA's exact sum: its folded 128-bit sum plus what
                    // the records still hold, converted once
                    unsigned long long lo, hi;
                    fold_bin(p, wp, b, lo, hi);
                    unsigned long long *f = p.wfold_buf + ((size_t)blockIdx.x * p.nbins + b) * 2;
                    const unsigned long long l1 = lo + f[0];
                    hi += f[1] + (l1 < lo ? 1ull : 0ull);
                    lo = l1;
                    f[0] = f[1] = 0ull;
                    w = ((double)hi * 18446744073709551616.0 + (double)lo) * wscale;
                } else if (p.wint) {
                    // per lane copy: the exact sum of its products (below
                    // 2^64) from its record of three 16-bit-piece sums
                    for (int k = 0; k < WK; ++k) {
                        const size_t e = ((size_t)b * WK + k) * 3;
                        const unsigned long long lo = (unsigned)take_i32<G>((int *)&wp[e]);
                        const unsigned long long mid = (unsigned)take_i32<G>((int *)&wp[e + 1]);
                        const unsigned long long hi = (unsigned)take_i32<G>((int *)&wp[e + 2]);
                        w += (double)(lo + (mid << 16) + (hi << 32));
                    }
                    w *= wscale;
                } else {
                    // binary64 sums, exchanged as their bit patterns
                    for (int k = 0; k < K; ++k)
                        w += __longlong_as_double((long long)take_u64<G>(&u[b * K + k]));
                }
                if (w != 0.0) atomicAdd(&p.whist[(size_t)h * p.nbins + b], w);
            }
        }
    }
    gsync<G>();
}

// ---------------------------------------------------------------------------
// FP32 binning of one in-range candidate
// ---------------------------------------------------------------------------
// Reciprocal square root: one MUFU.RSQ (PTX rsqrt.approx.ftz.f32, documented
// maximum relative error 2^-22.9; the rescue bands budget 2^-22).  +0 gives
// +inf, so coincident points produce NaN separations and are rescued.
// Base-2 logarithm: one MUFU.LG2 (PTX lg2.approx.ftz.f32).  Its error, at
// most 2.3e-7 max(1, |log2 x|) over every positive normal binary32 input
// (measured exhaustively; the log-bin bands budget 2^-21 max(1, |log2 x|)),
// is checked on the device by the test suite.  +0 gives -inf.
__device__ __forceinline__ float lg2_fast(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_fast(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Binning scalars, read from the kernel parameters once and kept in registers.
struct BinCtx {
    const float2 *lutA, *lutB;   // tables in shared memory
    float invA, invB;            // table cells per unit
    unsigned TA1, TB1;           // index of each table's sentinel cell
    float epsA, epsB;            // rescue bands of the two binned quantities
    float muA, muB, muW;         // mu band = muA / s + muB, table window muW
    unsigned nA, nB;
};

struct Bin32 {
    int bin;     // histogram index, valid only if ok
    bool ok;     // falls inside the histogram
    bool near;   // within an error band: needs the binary64 definition
};

__device__ __forceinline__ void lut_locate(const float2 *lut, float inv, unsigned t1, float v,
                                           int &k, float &edge) {
    // v >= 0 by construction; the unsigned clamp also sends any negative
    // index to the always-rescue sentinel cell
    unsigned t = min((unsigned)lut_index(v, inv), t1);
    float2 e = lut[t];
    edge = e.x;
    k = __float_as_int(e.y) + (v >= e.x ? 1 : 0);
}

// Within eps of the table edge (a NaN edge -- several edges in the cell's
// window -- always counts as near).
__device__ __forceinline__ bool is_near(float v, float e, float eps) {
    return !(fabsf(v - e) >= eps);
}

template <int MODE, int LOS>
__device__ __forceinline__ Bin32 bin_f32(const BinCtx &c, float dx, float dy, float dz,
                                         float qxy, float s2, float ax_, float ay_, float az_) {
    Bin32 r;
    if (MODE == MODE_S) {
        float rs = rsqrt_fast(s2);
        float s = s2 * rs;
        int k; float e;
        lut_locate(c.lutA, c.invA, c.TA1, s, k, e);
        r.near = is_near(s, e, c.epsA);
        r.ok = (unsigned)k < c.nA;
        r.bin = k;
        return r;
    }
    if (LOS == LOS_Z) {
        if (MODE == MODE_SMU) {
            float rs = rsqrt_fast(s2);
            float s = s2 * rs;
            float mu = fabsf(dz) * rs;
            int k, j; float e, em;
            lut_locate(c.lutA, c.invA, c.TA1, s, k, e);
            lut_locate(c.lutB, c.invB, c.TB1, mu, j, em);
            float epsm = fmaf(c.muA, rs, c.muB);
            r.near = is_near(s, e, c.epsA) || is_near(mu, em, epsm) || (epsm > c.muW);
            r.ok = (unsigned)k < c.nA;
            r.bin = k * (int)c.nB + j;
            return r;
        }
        // (sigma, pi) along z
        float sg = qxy * rsqrt_fast(qxy);
        float pz = fabsf(dz);
        int k, j; float e, ep;
        lut_locate(c.lutA, c.invA, c.TA1, sg, k, e);
        lut_locate(c.lutB, c.invB, c.TB1, pz, j, ep);
        r.near = is_near(sg, e, c.epsA) || is_near(pz, ep, c.epsB);
        r.ok = ((unsigned)k < c.nA) && ((unsigned)j < c.nB);
        r.bin = k * (int)c.nB + j;
        return r;
    }
    // midpoint line of sight: l = 2 x_i + d
    float lx = fmaf(2.0f, ax_, dx), ly = fmaf(2.0f, ay_, dy), lz = fmaf(2.0f, az_, dz);
    float sl = fmaf(dz, lz, fmaf(dy, ly, dx * lx));
    float ll = fmaf(lz, lz, fmaf(ly, ly, lx * lx));
    float rl = rsqrt_fast(ll);
    float pi = fabsf(sl) * rl;
    if (MODE == MODE_SMU) {
        float rs = rsqrt_fast(s2);
        float s = s2 * rs;
        float mu = pi * rs;
        int k, j; float e, em;
        lut_locate(c.lutA, c.invA, c.TA1, s, k, e);
        lut_locate(c.lutB, c.invB, c.TB1, mu, j, em);
        float epsm = fmaf(c.muA, rs, c.muB);
        r.near = is_near(s, e, c.epsA) || is_near(mu, em, epsm) || (epsm > c.muW);
        r.ok = (unsigned)k < c.nA;
        r.bin = k * (int)c.nB + j;
        return r;
    }
    // sigma = |d x l| / |l|
    float cxp = fmaf(dy, lz, -dz * ly);
    float cyp = fmaf(dz, lx, -dx * lz);
    float czp = fmaf(dx, ly, -dy * lx);
    float cc = fmaf(czp, czp, fmaf(cyp, cyp, cxp * cxp));
    float sg = cc * rsqrt_fast(cc) * rl;
    int k, j; float e, ep;
    lut_locate(c.lutA, c.invA, c.TA1, sg, k, e);
    lut_locate(c.lutB, c.invB, c.TB1, pi, j, ep);
    r.near = is_near(sg, e, c.epsA) || is_near(pi, ep, c.epsB);
    r.ok = ((unsigned)k < c.nA) && ((unsigned)j < c.nB);
    r.bin = k * (int)c.nB + j;
    return r;
}

// Evenly spaced s bins (and mu bins for (s, mu) along z): bin = floor of a
// scaled value; the pair is near an edge when that value's fractional part
// is within the band of 0 or 1.
struct LinCtx {
    float invA, offA, thrA;   // s scaling and band threshold
    float mS;                 // logarithmic s: band term per 1/s
    float invB2, thrB;        // (sigma, pi): pi scaling and band threshold
    float nB, mA, cB;         // mu scaling and per-pair band threshold
    unsigned nA, nB_u;
};



// Shared-memory reduction at a 32-bit shared-window address, issued only
// when `on` is set (one predicated instruction, no branch).
__device__ __forceinline__ void red_shared_u32_if(unsigned addr, bool on) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t@p red.shared.add.u32 [%0], 1;\n\t}"
        ::"r"(addr), "r"((unsigned)on));
}
// Unpredicated: the whole warp issues it, lanes without a pair pointing at
// the discarded row.  A partially predicated shared reduction measured about
// half the throughput of a full-warp one on this GPU.
__device__ __forceinline__ void red_shared_u32(unsigned addr, unsigned v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
// The three 16-bit pieces of an integer weight product p = P >> 16 into one
// lane copy's record {lo, mid, hi} (immediate offsets from one address),
// taken from the 64-bit product P itself: bits 16-31, 32-47 and 48-63.
__device__ __forceinline__ void red_shared_pieces(unsigned addr, unsigned long long P) {
    const unsigned lo = (unsigned)P, hi = (unsigned)(P >> 32);
    asm volatile(
        "red.shared.add.u32 [%0], %1;\n\t"
        "red.shared.add.u32 [%0+4], %2;\n\t"
        "red.shared.add.u32 [%0+8], %3;" ::"r"(addr),
        "r"(lo >> 16), "r"(hi & 0xFFFFu), "r"(hi >> 16));
}
// Integer weight product of a pair with binary64 remainders (W == 3), in
// units of the task's wscale: V = round(P / 2^16 + c) with P the exact
// product of the packed weights (hi_i hi_j = P 2^-16 wscale) and c the
// remainder terms (hi_i lo_j + lo_i hi_j) / wscale = pf_i l_j + l_i pf_j (l
// the scaled remainders, pf the packed weights as binary32), evaluated in
// binary32 (|c| < 2^-23 P / 2^16 < 2^25) and rounded to an integer.  V is
// non-negative and below 2^49; its error against the exact w_i w_j / wscale
// is at most 1 + 2^-40 P / 2^16 units (the two roundings, the dropped
// lo_i lo_j and the binary32 error of c).
__device__ __forceinline__ unsigned long long corrected_product(unsigned wi, float pfi, float li,
                                                                unsigned wj, float lj) {
    const float c = fmaf(pfi, lj, li * __uint2float_rn(wj));
    const long long k = (long long)__float2int_rn(c);
    const unsigned long long P = (unsigned long long)wi * wj;
    return ((P + 0x8000ull) >> 16) + (unsigned long long)k;
}
// The three pieces of V (bits 0-15, 16-31 and 32-48) into one lane copy's
// record, as red_shared_pieces does for P >> 16.
__device__ __forceinline__ void red_shared_pieces_v(unsigned addr, unsigned long long V) {
    const unsigned lo = (unsigned)V, hi = (unsigned)(V >> 32);
    asm volatile(
        "red.shared.add.u32 [%0], %1;\n\t"
        "red.shared.add.u32 [%0+4], %2;\n\t"
        "red.shared.add.u32 [%0+8], %3;" ::"r"(addr),
        "r"(lo & 0xFFFFu), "r"(lo >> 16), "r"(hi));
}
__device__ __forceinline__ void red_shared_f64_if(unsigned addr, double v, bool on) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p red.shared.add.f64 [%0], %1;\n\t}"
        ::"r"(addr), "d"(v), "r"((unsigned)on));
}

// Rare path: stage one near-edge pair for the binary64 rescue.
template <int MODE, int LOS>
__device__ __noinline__ void rescue_push(const PairParams &p, uint3 *s_q, int *s_qn,
                                         const int4 *s_seg, int nseg, int f0, int fstride, int jj,
                                         int bstart, int i, unsigned task_bits) {
    int jidx, img;
    if (f0 < 0) {
        jidx = bstart + jj;
        img = 13;
    } else {
        // tile f0 holds the chunk's j-groups f0, f0 + fstride, f0 + 2 fstride, ...
        const int f = ((jj / JG) * fstride + f0) * JG + (jj % JG);
        int4 sg = s_seg[seg_find(s_seg, nseg, f)];
        jidx = sg.x + (f - sg.y);
        img = sg.w;
    }
    push_rescue<MODE, LOS>(p, s_q, s_qn,
                           make_uint3((unsigned)i, (unsigned)jidx, (unsigned)img | task_bits));
}

// Everything the inner loop needs, in registers.
template <int RI>
struct IPts {
    float x[RI], y[RI], z[RI];     // offsets from the i-cell centre (far away if unused)
    float xa[RI], ya[RI], za[RI];  // absolute positions (midpoint line of sight)
    double w[RI];
    unsigned wm[RI];               // packed integer weight (integer weight path)
    float wl[RI], pf[RI];          // W == 3: scaled remainder, packed weight as binary32
    int idx[RI];
};

// A staged tile of j-points (structure of arrays, even length, shifted into
// the i-cell's frame).
struct Tile {
    const float *x, *y, *z;
    const double *w;               // binary64 weights (W == 1)
    const unsigned *wm;            // packed integer weights (W >= 2), same storage
    const float *wl;               // scaled binary64 remainders (W == 3), after wm
};

// Table-based bins, one pair at a time (every mode and line of sight).
// MASK: the tile holds the block's own points and only pairs j > i count.
template <int MODE, int LOS, int W, int RI, bool MASK>
__device__ __forceinline__ void pair_tile_lut(const PairParams &p, Tile tb, int len, unsigned gmask,
                                              const IPts<RI> &I, const BinCtx &bc, float r2cut,
                                              unsigned hist_sa, unsigned whist_sa, unsigned hk4,
                                              uint3 *s_q, int *s_qn, const int4 *s_seg, int nseg,
                                              int f0, int fstride, int bstart, unsigned task_bits) {
#pragma unroll 1
    for (unsigned gm = gmask; gm; gm &= gm - 1) {
    const int j0 = (__ffs(gm) - 1) * JG, j1 = min(j0 + JG, len);
#pragma unroll 2
    for (int jj = j0; jj < j1; ++jj) {
        const float qx = tb.x[jj], qy = tb.y[jj], qz = tb.z[jj];
        float dxv[RI], dyv[RI], dzv[RI], qv[RI], s2v[RI];
        bool inr[RI];
        bool any = false;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            dxv[r] = qx - I.x[r];
            dyv[r] = qy - I.y[r];
            dzv[r] = qz - I.z[r];
            qv[r] = fmaf(dyv[r], dyv[r], dxv[r] * dxv[r]);
            s2v[r] = fmaf(dzv[r], dzv[r], qv[r]);
            inr[r] = s2v[r] < r2cut;
            if (MASK) inr[r] = inr[r] && (bstart + jj > I.idx[r]);
            any = any || inr[r];
        }
        if (__any_sync(0xffffffffu, any)) {
            double wj = 0.0;
            if (W == 1) wj = tb.w[jj];
            bool resc[RI];
            bool anyr = false;
#pragma unroll
            for (int r = 0; r < RI; ++r) {
                Bin32 b = bin_f32<MODE, LOS>(bc, dxv[r], dyv[r], dzv[r], qv[r], s2v[r], I.xa[r],
                                             I.ya[r], I.za[r]);
                const bool add = inr[r] && b.ok && !b.near;
                red_shared_u32_if(hist_sa + hk4 * (unsigned)b.bin, add);
                if (W == 1) red_shared_f64_if(whist_sa + 2u * hk4 * (unsigned)b.bin, __dmul_rn(I.w[r], wj), add);
                resc[r] = inr[r] && b.near;
                anyr = anyr || resc[r];
            }
            if (__any_sync(0xffffffffu, anyr)) {
#pragma unroll
                for (int r = 0; r < RI; ++r)
                    if (resc[r])
                        rescue_push<MODE, LOS>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj, bstart, I.idx[r],
                                               task_bits);
            }
        }
    }
    }
}

// Evenly spaced bins, two j-points per step in packed FP32 (s, and (s, mu)
// along z).  For each pair: t_s = (s - e0) / D, bin = floor(t_s); the pair
// is near an edge unless |frac(t_s) - 1/2| < thrA; mu likewise with its
// per-pair band.  Histogram addresses are formed from the float bits of
// floor(t) + 2^23, with the 2^23 bias folded into the base address.
template <int MODE, int W, int RI, bool MASK, bool CHK, bool LOGS>
__device__ __forceinline__ void pair_tile_lin2(const PairParams &p, Tile tb, int len, unsigned gmask,
                                               const IPts<RI> &I, const LinCtx &lc, float r2cut,
                                               unsigned hist_sa, unsigned whist_sa, unsigned hk4,
                                               uint3 *s_q, int *s_qn, const int4 *s_seg, int nseg,
                                               int f0, int fstride, int bstart, unsigned task_bits) {
    const float2 C23 = make_float2(8388608.0f, 8388608.0f);
    const float2 NC23H = make_float2(-8388608.0f + 0.5f, -8388608.0f + 0.5f);
    const float2 M1 = make_float2(-1.0f, -1.0f);
    const float2 INVA = make_float2(lc.invA, lc.invA);
    const float2 OFFA = make_float2(lc.offA, lc.offA);
    const float2 NB = make_float2(lc.nB, lc.nB);
    const float2 NMA = make_float2(-lc.mA, -lc.mA);
    const float2 CB = make_float2(lc.cB, lc.cB);
    // With the range test (CHK) the offset carries +1 (host side): t_s + 1 >= 0
    // for every t_s >= -1, where adding 2^23 and rounding down is an exact
    // floor (below 2^23 the float spacing is 1/2); values below -1 are out of
    // range whatever their floor.  The extra row is removed in the base.
    const float halfA = 0.5f * (float)lc.nA;
    const float hA1 = CHK ? halfA + 1.0f : halfA;
    const float2 NHALFA = make_float2(-hA1, -hA1);
    const float thrA = lc.thrA;
    const float2 THRA = make_float2(lc.thrA, lc.thrA);
    const float2 NMS = make_float2(-lc.mS, -lc.mS);
    const unsigned nbu = (MODE == MODE_SMU) ? lc.nB_u : 1u;
    // biases of the float bits of floor(t_s) + 2^23 (and floor(t_mu) + 2^23),
    // folded into the bases
    const unsigned bias = 0x4B000000u * nbu + ((MODE == MODE_SMU) ? 0x4B000000u : 0u) +
                          (CHK ? nbu : 0u);
    const unsigned hbase = hist_sa - hk4 * bias;
    const unsigned htrash = hist_sa + hk4 * (unsigned)p.trash_row;
    const unsigned wbase = whist_sa - 2u * hk4 * bias;
    // integer weights: a 12-byte record {lo, mid, hi} per bin and lane copy
    // (word 3 (bin copies + copy) + piece: bank 3 copy + piece, conflict-free),
    // as many copies as the counts, so a record's address is 3 x the count's
    // address + wdelta (the discarded row included)
    const unsigned wdelta = whist_sa - 3u * hist_sa;
    float2 NX[RI], NY[RI], NZ[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        NX[r] = make_float2(-I.x[r], -I.x[r]);
        NY[r] = make_float2(-I.y[r], -I.y[r]);
        NZ[r] = make_float2(-I.z[r], -I.z[r]);
    }
#pragma unroll 1
    for (unsigned gm = gmask; gm; gm &= gm - 1) {
    const int j0 = (__ffs(gm) - 1) * JG, j1 = min(j0 + JG, len);
#pragma unroll 4
    for (int jj = j0; jj < j1; jj += 2) {
        const float2 X = *reinterpret_cast<const float2 *>(tb.x + jj);
        const float2 Y = *reinterpret_cast<const float2 *>(tb.y + jj);
        const float2 Z = *reinterpret_cast<const float2 *>(tb.z + jj);
        float2 S2[RI], DZ[RI];
        bool in0[RI], in1[RI];
        bool any = false;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const float2 dx = __fadd2_rn(X, NX[r]);
            const float2 dy = __fadd2_rn(Y, NY[r]);
            DZ[r] = __fadd2_rn(Z, NZ[r]);
            S2[r] = __ffma2_rn(DZ[r], DZ[r], __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            in0[r] = S2[r].x < r2cut;
            in1[r] = S2[r].y < r2cut;
            if (MASK) {
                in0[r] = in0[r] && (bstart + jj > I.idx[r]);
                in1[r] = in1[r] && (bstart + jj + 1 > I.idx[r]);
            }
            any = any || in0[r] || in1[r];
        }
        if (__any_sync(0xffffffffu, any)) {
            bool re0[RI], re1[RI];
            bool anyr = false;
#pragma unroll
            for (int r = 0; r < RI; ++r) {
                const float2 s2 = S2[r];
                const float2 rs = make_float2(rsqrt_fast(s2.x), rsqrt_fast(s2.y));
                // t_s = (s - e0) / D, or log_q(s / e0) = A log2(s^2) + B
                const float2 ts =
                    LOGS ? __ffma2_rn(make_float2(lg2_fast(s2.x), lg2_fast(s2.y)), INVA, OFFA)
                         : __ffma2_rn(__fmul2_rn(s2, rs), INVA, OFFA);
                const float2 f = __fadd2_rd(ts, C23);
                const float2 d = __ffma2_rn(__fadd2_rn(f, NC23H), M1, ts);   // frac - 1/2
                bool ok0 = true, ok1 = true;
                if (CHK) {
                    const float2 o = __fadd2_rn(ts, NHALFA);
                    ok0 = fabsf(o.x) < halfA;
                    ok1 = fabsf(o.y) < halfA;
                }
                // NaN (s2 = 0) compares false: such pairs are near.  Log edges:
                // the band grows as 1/s
                const float2 ths = LOGS ? __ffma2_rn(NMS, rs, THRA) : THRA;
                bool n0 = !(fabsf(d.x) < ths.x), n1 = !(fabsf(d.y) < ths.y);
                unsigned b0 = (unsigned)__float_as_int(f.x), b1 = (unsigned)__float_as_int(f.y);
                if (MODE == MODE_SMU) {
                    const float2 adz = make_float2(fabsf(DZ[r].x), fabsf(DZ[r].y));
                    const float2 tm = __fmul2_rn(adz, __fmul2_rn(rs, NB));
                    const float2 fm = __fadd2_rd(tm, C23);
                    const float2 dm = __ffma2_rn(__fadd2_rn(fm, NC23H), M1, tm);
                    const float2 thm = __ffma2_rn(NMA, rs, CB);
                    n0 = n0 || !(fabsf(dm.x) < thm.x);
                    n1 = n1 || !(fabsf(dm.y) < thm.y);
                    // t_mu < n_mu (scale below n_mu): mu = 1 is in the last bin;
                    // a NaN index is never used (such pairs are near)
                    const unsigned j0 = (unsigned)__float_as_int(fm.x);
                    const unsigned j1 = (unsigned)__float_as_int(fm.y);
                    b0 = b0 * nbu + j0;
                    b1 = b1 * nbu + j1;
                }
                const bool a0 = in0[r] && ok0 && !n0, a1 = in1[r] && ok1 && !n1;
                const unsigned c0 = a0 ? hbase + hk4 * b0 : htrash;
                const unsigned c1 = a1 ? hbase + hk4 * b1 : htrash;
                red_shared_u32(c0, 1u);
                red_shared_u32(c1, 1u);
                if (W == 1) {
                    const double2 wj = *reinterpret_cast<const double2 *>(tb.w + jj);
                    red_shared_f64_if(wbase + 2u * hk4 * b0, __dmul_rn(I.w[r], wj.x), a0);
                    red_shared_f64_if(wbase + 2u * hk4 * b1, __dmul_rn(I.w[r], wj.y), a1);
                } else if (W == 2) {
                    // (M_i M_j) >> (k_i + k_j), k = emax - e the exponent offset:
                    // the packed M 2^(8 - k) multiplied exactly in 64 bits is
                    // P = M_i M_j 2^(16 - k_i - k_j), and the product is P >> 16
                    // (truncation < 2^(k_i + k_j - 46) relative, below 2^48),
                    // added as three 16-bit pieces to the lane copy's record
                    const uint2 wj = *reinterpret_cast<const uint2 *>(tb.wm + jj);
                    red_shared_pieces(3u * c0 + wdelta, (unsigned long long)I.wm[r] * wj.x);
                    red_shared_pieces(3u * c1 + wdelta, (unsigned long long)I.wm[r] * wj.y);
                } else if (W == 3) {
                    // the same product with the binary64 remainders' terms
                    const uint2 wj = *reinterpret_cast<const uint2 *>(tb.wm + jj);
                    const float2 lj = *reinterpret_cast<const float2 *>(tb.wl + jj);
                    red_shared_pieces_v(3u * c0 + wdelta,
                                        corrected_product(I.wm[r], I.pf[r], I.wl[r], wj.x, lj.x));
                    red_shared_pieces_v(3u * c1 + wdelta,
                                        corrected_product(I.wm[r], I.pf[r], I.wl[r], wj.y, lj.y));
                }
                re0[r] = in0[r] && n0;
                re1[r] = in1[r] && n1;
                anyr = anyr || re0[r] || re1[r];
            }
            if (__any_sync(0xffffffffu, anyr)) {
#pragma unroll
                for (int r = 0; r < RI; ++r) {
                    if (re0[r])
                        rescue_push<MODE, LOS_Z>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj, bstart,
                                                 I.idx[r], task_bits);
                    if (re1[r])
                        rescue_push<MODE, LOS_Z>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj + 1, bstart,
                                                 I.idx[r], task_bits);
                }
            }
        }
    }
    }
}

// (sigma, pi) bins, both axes evenly spaced from 0, two j-points per step in
// packed FP32.  sigma and pi are formed exactly as in the table path (so the
// same bands apply): along z, sigma = q rsqrt(q) with q = dx^2 + dy^2 and
// pi = |dz|; for the midpoint line of sight l = 2 x_i + d, pi = |d.l| / |l|
// and sigma = |d x l| / |l|.  Both indices are floors on the 2^23 grid; the
// pair counts only if both lie below their axis' bin count (pi may exceed
// pi_max while s is still below the reach sqrt(sigma_max^2 + pi_max^2)).
template <int LOS, int W, int RI, bool MASK>
__device__ __forceinline__ void pair_tile_sigpi2(const PairParams &p, Tile tb, int len, unsigned gmask,
                                                 const IPts<RI> &I, const LinCtx &lc, float r2cut,
                                                 unsigned hist_sa, unsigned whist_sa, unsigned hk4,
                                                 uint3 *s_q, int *s_qn, const int4 *s_seg, int nseg,
                                                 int f0, int fstride, int bstart,
                                                 unsigned task_bits) {
    const float2 C23 = make_float2(8388608.0f, 8388608.0f);
    const float2 NC23H = make_float2(-8388608.0f + 0.5f, -8388608.0f + 0.5f);
    const float2 M1 = make_float2(-1.0f, -1.0f);
    const float2 TWO = make_float2(2.0f, 2.0f);
    const float2 INVA = make_float2(lc.invA, lc.invA);
    const float2 INVB = make_float2(lc.invB2, lc.invB2);
    const float thrA = lc.thrA, thrB = lc.thrB;
    const unsigned nbu = lc.nB_u;
    const unsigned limA = 0x4B000000u + lc.nA, limB = 0x4B000000u + lc.nB_u;
    const unsigned bias = 0x4B000000u * nbu + 0x4B000000u;
    const unsigned hbase = hist_sa - hk4 * bias;
    const unsigned htrash = hist_sa + hk4 * (unsigned)p.trash_row;
    const unsigned wbase = whist_sa - 2u * hk4 * bias;
    const unsigned wdelta = whist_sa - 3u * hist_sa;   // as in the floor-bin loop above
    float2 NX[RI], NY[RI], NZ[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        NX[r] = make_float2(-I.x[r], -I.x[r]);
        NY[r] = make_float2(-I.y[r], -I.y[r]);
        NZ[r] = make_float2(-I.z[r], -I.z[r]);
    }
#pragma unroll 1
    for (unsigned gm = gmask; gm; gm &= gm - 1) {
    const int j0 = (__ffs(gm) - 1) * JG, j1 = min(j0 + JG, len);
#pragma unroll 2
    for (int jj = j0; jj < j1; jj += 2) {
        const float2 X = *reinterpret_cast<const float2 *>(tb.x + jj);
        const float2 Y = *reinterpret_cast<const float2 *>(tb.y + jj);
        const float2 Z = *reinterpret_cast<const float2 *>(tb.z + jj);
        float2 S2[RI];
        bool in0[RI], in1[RI];
        bool any = false;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const float2 dx = __fadd2_rn(X, NX[r]);
            const float2 dy = __fadd2_rn(Y, NY[r]);
            const float2 dz = __fadd2_rn(Z, NZ[r]);
            S2[r] = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            in0[r] = S2[r].x < r2cut;
            in1[r] = S2[r].y < r2cut;
            if (MASK) {
                in0[r] = in0[r] && (bstart + jj > I.idx[r]);
                in1[r] = in1[r] && (bstart + jj + 1 > I.idx[r]);
            }
            any = any || in0[r] || in1[r];
        }
        if (__any_sync(0xffffffffu, any)) {
            bool re0[RI], re1[RI];
            bool anyr = false;
#pragma unroll
            for (int r = 0; r < RI; ++r) {
                const float2 dx = __fadd2_rn(X, NX[r]);
                const float2 dy = __fadd2_rn(Y, NY[r]);
                const float2 dz = __fadd2_rn(Z, NZ[r]);
                float2 sg, pz;
                if (LOS == LOS_Z) {
                    const float2 q = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
                    sg = __fmul2_rn(q, make_float2(rsqrt_fast(q.x), rsqrt_fast(q.y)));
                    pz = make_float2(fabsf(dz.x), fabsf(dz.y));
                } else {
                    const float2 lx = __ffma2_rn(TWO, make_float2(I.xa[r], I.xa[r]), dx);
                    const float2 ly = __ffma2_rn(TWO, make_float2(I.ya[r], I.ya[r]), dy);
                    const float2 lz = __ffma2_rn(TWO, make_float2(I.za[r], I.za[r]), dz);
                    const float2 sl = __ffma2_rn(dz, lz, __ffma2_rn(dy, ly, __fmul2_rn(dx, lx)));
                    const float2 ll = __ffma2_rn(lz, lz, __ffma2_rn(ly, ly, __fmul2_rn(lx, lx)));
                    const float2 rl = make_float2(rsqrt_fast(ll.x), rsqrt_fast(ll.y));
                    pz = __fmul2_rn(make_float2(fabsf(sl.x), fabsf(sl.y)), rl);
                    const float2 ndx = make_float2(-dx.x, -dx.y), ndy = make_float2(-dy.x, -dy.y),
                                 ndz = make_float2(-dz.x, -dz.y);
                    const float2 cx = __ffma2_rn(dy, lz, __fmul2_rn(ndz, ly));
                    const float2 cy = __ffma2_rn(dz, lx, __fmul2_rn(ndx, lz));
                    const float2 cz = __ffma2_rn(dx, ly, __fmul2_rn(ndy, lx));
                    const float2 cc = __ffma2_rn(cz, cz, __ffma2_rn(cy, cy, __fmul2_rn(cx, cx)));
                    sg = __fmul2_rn(__fmul2_rn(cc, make_float2(rsqrt_fast(cc.x), rsqrt_fast(cc.y))), rl);
                }
                const float2 ta = __fmul2_rn(sg, INVA), tb2 = __fmul2_rn(pz, INVB);
                const float2 fa = __fadd2_rd(ta, C23), fb = __fadd2_rd(tb2, C23);
                const float2 da = __ffma2_rn(__fadd2_rn(fa, NC23H), M1, ta);   // frac - 1/2
                const float2 db = __ffma2_rn(__fadd2_rn(fb, NC23H), M1, tb2);
                // NaN (s = 0 or l = 0) compares false: near
                const bool n0 = !(fabsf(da.x) < thrA) || !(fabsf(db.x) < thrB);
                const bool n1 = !(fabsf(da.y) < thrA) || !(fabsf(db.y) < thrB);
                const unsigned ba0 = (unsigned)__float_as_int(fa.x), ba1 = (unsigned)__float_as_int(fa.y);
                const unsigned bb0 = (unsigned)__float_as_int(fb.x), bb1 = (unsigned)__float_as_int(fb.y);
                const bool ok0 = ba0 < limA && bb0 < limB, ok1 = ba1 < limA && bb1 < limB;
                const unsigned b0 = ba0 * nbu + bb0, b1 = ba1 * nbu + bb1;
                const bool a0 = in0[r] && ok0 && !n0, a1 = in1[r] && ok1 && !n1;
                const unsigned c0 = a0 ? hbase + hk4 * b0 : htrash;
                const unsigned c1 = a1 ? hbase + hk4 * b1 : htrash;
                red_shared_u32(c0, 1u);
                red_shared_u32(c1, 1u);
                if (W == 1) {
                    const double2 wj = *reinterpret_cast<const double2 *>(tb.w + jj);
                    red_shared_f64_if(wbase + 2u * hk4 * b0, __dmul_rn(I.w[r], wj.x), a0);
                    red_shared_f64_if(wbase + 2u * hk4 * b1, __dmul_rn(I.w[r], wj.y), a1);
                } else if (W == 2) {
                    const uint2 wj = *reinterpret_cast<const uint2 *>(tb.wm + jj);
                    red_shared_pieces(3u * c0 + wdelta, (unsigned long long)I.wm[r] * wj.x);
                    red_shared_pieces(3u * c1 + wdelta, (unsigned long long)I.wm[r] * wj.y);
                } else if (W == 3) {
                    const uint2 wj = *reinterpret_cast<const uint2 *>(tb.wm + jj);
                    const float2 lj = *reinterpret_cast<const float2 *>(tb.wl + jj);
                    red_shared_pieces_v(3u * c0 + wdelta,
                                        corrected_product(I.wm[r], I.pf[r], I.wl[r], wj.x, lj.x));
                    red_shared_pieces_v(3u * c1 + wdelta,
                                        corrected_product(I.wm[r], I.pf[r], I.wl[r], wj.y, lj.y));
                }
                re0[r] = in0[r] && n0;
                re1[r] = in1[r] && n1;
                anyr = anyr || re0[r] || re1[r];
            }
            if (__any_sync(0xffffffffu, anyr)) {
#pragma unroll
                for (int r = 0; r < RI; ++r) {
                    if (re0[r])
                        rescue_push<MODE_SIGPI, LOS>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj,
                                                     bstart, I.idx[r], task_bits);
                    if (re1[r])
                        rescue_push<MODE_SIGPI, LOS>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj + 1,
                                                     bstart, I.idx[r], task_bits);
                }
            }
        }
    }
    }
}

// Global-histogram variant for histograms too large for shared memory.
template <int MODE, int LOS, int W, int RI, bool MASK>
__device__ __forceinline__ void pair_tile_global(const PairParams &p, Tile tb, int len, unsigned gmask,
                                                 const IPts<RI> &I, const BinCtx &bc, float r2cut,
                                                 size_t hbase, uint3 *s_q, int *s_qn,
                                                 const int4 *s_seg, int nseg, int f0, int fstride, int bstart,
                                                 unsigned task_bits) {
    for (unsigned gm = gmask; gm; gm &= gm - 1) {
    const int j0 = (__ffs(gm) - 1) * JG, j1 = min(j0 + JG, len);
    for (int jj = j0; jj < j1; ++jj) {
        const float qx = tb.x[jj], qy = tb.y[jj], qz = tb.z[jj];
        for (int r = 0; r < RI; ++r) {
            float dx = qx - I.x[r], dy = qy - I.y[r], dz = qz - I.z[r];
            float qxy = fmaf(dy, dy, dx * dx);
            float s2 = fmaf(dz, dz, qxy);
            bool inr = s2 < r2cut;
            if (MASK) inr = inr && (bstart + jj > I.idx[r]);
            if (!inr) continue;
            Bin32 b = bin_f32<MODE, LOS>(bc, dx, dy, dz, qxy, s2, I.xa[r], I.ya[r], I.za[r]);
            if (b.near) {
                rescue_push<MODE, LOS>(p, s_q, s_qn, s_seg, nseg, f0, fstride, jj, bstart, I.idx[r],
                                       task_bits);
            } else if (b.ok) {
                atomicAdd(p.hist + hbase + b.bin, 1ull);
                if (W == 1) atomicAdd(p.whist + hbase + b.bin, __dmul_rn(I.w[r], tb.w[jj]));
            }
        }
    }
    }
}

// One tile through the variant that applies.
template <int MODE, int LOS, int W, int RI, bool LIN, bool MASK>
__device__ __forceinline__ void pair_tile(const PairParams &p, bool smem_hist, Tile tb, int len,
                                          unsigned gmask,
                                          const IPts<RI> &I, const BinCtx &bc, const LinCtx &lc,
                                          float r2cut, unsigned hist_sa, unsigned whist_sa,
                                          unsigned hk4, size_t hbase, uint3 *s_q, int *s_qn,
                                          const int4 *s_seg,
                                          int nseg, int f0, int fstride, int bstart, unsigned task_bits) {
    static_assert(W < 2 || LIN, "integer weights run only with floor-based bins");
    if (!smem_hist) {
        pair_tile_global<MODE, LOS, W, RI, MASK>(p, tb, len, gmask, I, bc, r2cut, hbase, s_q, s_qn, s_seg,
                                                 nseg, f0, fstride, bstart, task_bits);
    } else if constexpr (LIN && MODE == MODE_SIGPI) {
        pair_tile_sigpi2<LOS, W, RI, MASK>(p, tb, len, gmask, I, lc, r2cut, hist_sa, whist_sa, hk4,
                                           s_q, s_qn, s_seg, nseg, f0, fstride, bstart, task_bits);
    } else if constexpr (LIN) {
        if (p.lin_log)
            pair_tile_lin2<MODE, W, RI, MASK, true, true>(p, tb, len, gmask, I, lc, r2cut, hist_sa,
                                                          whist_sa, hk4, s_q, s_qn, s_seg, nseg,
                                                          f0, fstride, bstart, task_bits);
        else if (p.lin_norange)
            pair_tile_lin2<MODE, W, RI, MASK, false, false>(p, tb, len, gmask, I, lc, r2cut, hist_sa,
                                                     whist_sa, hk4, s_q, s_qn, s_seg, nseg, f0, fstride,
                                                     bstart, task_bits);
        else
            pair_tile_lin2<MODE, W, RI, MASK, true, false>(p, tb, len, gmask, I, lc, r2cut, hist_sa,
                                                    whist_sa, hk4, s_q, s_qn,
                                          s_seg, nseg, f0, fstride, bstart, task_bits);
    } else {
        pair_tile_lut<MODE, LOS, W, RI, MASK>(p, tb, len, gmask, I, bc, r2cut, hist_sa, whist_sa,
                                              hk4, s_q,
                                              s_qn, s_seg, nseg, f0, fstride, bstart, task_bits);
    }
}

// ---------------------------------------------------------------------------
// FP32 kernel
// ---------------------------------------------------------------------------
// W: 0 unweighted, 1 binary64 weighted sums, 2 integer weight products.
// G: independent groups of NT threads per CTA that share the histograms (a
// large histogram then keeps G x 4 warps per SM busy instead of 4).
// TREE: blocks are k-d tree nodes and their j-segments come from the list of
// the dual-tree traversal instead of the stencil rows.
template <int MODE, int LOS, int W, int RI, bool LIN, int G = 1, bool TREE = false>
__global__ void __launch_bounds__(NT * G, (G > 1 ? 1 : (RI <= 2 ? 5 : 4)))
    k_pairs_f32(const __grid_constant__ PairParams p) {
    static_assert(!TREE || G == 1, "the tree variant runs one thread group per CTA");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CtaShared cs_g[G];
    __shared__ int s_tmp_g[G][8];
    __shared__ unsigned long long s_base_g[G];
    __shared__ GBox s_gbox_g[G][2][TJ / JG];   // bounding boxes of the staged j-groups
    __shared__ GBox s_ibox_g[G][NT / 32];      // bounding box of each warp's i-points
    const int grp = (int)(threadIdx.x / NT);
    CtaShared &cs = cs_g[grp];
    int *s_tmp = s_tmp_g[grp];
    unsigned long long &s_base = s_base_g[grp];
    GBox(*s_gbox)[TJ / JG] = s_gbox_g[grp];
    GBox *s_ibox = s_ibox_g[grp];

    const SmemLayout Ly = smem_layout(p, false);
    float2 *s_lut = (float2 *)(smem + Ly.lut);
    int *s_hist = (int *)(smem + Ly.hist);
    double *s_whist = (double *)(smem + Ly.whist);
    unsigned char *gsm = smem + (size_t)grp * Ly.gstride;   // this group's own area
    int4 *s_seg = (int4 *)(gsm + Ly.seg);
    float *s_tx = (float *)(gsm + Ly.tile);     // [2][TJ] each
    float *s_ty = s_tx + 2 * TJ;
    float *s_tz = s_ty + 2 * TJ;
    double *s_tw = (double *)(gsm + Ly.tw);
    unsigned *s_twm = (unsigned *)(gsm + Ly.tw);   // packed weights share the storage
    float *s_twl = (float *)(s_twm + 2 * TJ);      // W == 3: remainders after them
    uint3 *s_q = (uint3 *)(gsm + Ly.q);
    float4 *s_soff = (float4 *)(gsm + Ly.meta);   // tree: offset of each segment's block centre

    const int tid = gtid();
    for (int k = threadIdx.x; k < p.lut_total; k += NT * G) s_lut[k] = p.lut[k];
    const int nbins = p.nbins;
    const bool smem_hist = p.smem_hist_ok != 0;
    if (smem_hist) {
        const int copies = (p.priv ? NT / 32 : 1) * p.hist_k;
        for (int k = threadIdx.x; k < p.nbins_smem * copies; k += NT * G) s_hist[k] = 0;
        if (W >= 2) {   // the integer weight records (and this CTA's folded sums)
            unsigned *wp = reinterpret_cast<unsigned *>(s_whist);
            for (int k = threadIdx.x; k < 3 * p.nbins_smem * p.wint_k; k += NT * G) wp[k] = 0u;
            if (p.wfold)
                for (int b = threadIdx.x; b < p.nbins; b += NT) {
                    unsigned long long *f = p.wfold_buf + ((size_t)blockIdx.x * p.nbins + b) * 2;
                    f[0] = f[1] = 0ull;
                }
        } else if (W) {
            for (int k = threadIdx.x; k < p.nbins_smem * p.hist_k; k += NT * G) s_whist[k] = 0.0;
        }
    }
    if (tid == 0) {
        cs.qn = 0;
        cs.pruned = 0;
    }

    BinCtx bc;
    bc.lutA = s_lut + p.la.off;
    bc.lutB = s_lut + p.lb.off;
    bc.invA = p.la.inv_w;
    bc.invB = p.lb.inv_w;
    bc.TA1 = (unsigned)(p.la.T + 1);
    bc.TB1 = (unsigned)(p.lb.T + 1);
    bc.epsA = p.eps_a;
    bc.epsB = p.eps_b;
    bc.muA = p.mu_A;
    bc.muB = p.mu_B;
    bc.muW = p.mu_W;
    bc.nA = (unsigned)p.n_a;
    bc.nB = (unsigned)p.n_b;
    LinCtx lc;
    lc.invA = p.lin_invA;
    lc.offA = p.lin_offA;
    lc.thrA = p.lin_thrA;
    lc.mS = p.lin_mS;
    lc.invB2 = p.lin_invB2;
    lc.thrB = p.lin_thrB;
    lc.nB = p.lin_nB;
    lc.mA = p.lin_mA;
    lc.cB = p.lin_cB;
    lc.nA = (unsigned)p.n_a;
    lc.nB_u = (unsigned)p.n_b;
    const float r2cut = p.r2cut;
    // this thread's copy: warp copy (priv) and lane copy (tid % hist_k); bins
    // are hist_k entries apart
    const unsigned lane_copy = (unsigned)(tid & (p.hist_k - 1));
    const unsigned hk4 = 4u * (unsigned)p.hist_k;
    const unsigned hist_sa = (unsigned)__cvta_generic_to_shared(s_hist) +
                             (p.priv ? (unsigned)((tid >> 5) * p.nbins_smem * p.hist_k * 4) : 0u) +
                             4u * lane_copy;
    const unsigned whist_sa = (unsigned)__cvta_generic_to_shared(s_whist) +
                              (W >= 2 ? 12u * lane_copy : 8u * lane_copy);

    const int nx = p.g.ng[0], ny = p.g.ng[1];
    const float c32x = p.g.c32[0], c32y = p.g.c32[1], c32z = p.g.c32[2];
    const int nblocks = *p.nblocks;
    unsigned long long cand_local = 0;    // thread 0 only
    unsigned long long since_flush = 0;   // CTA-uniform
    unsigned long long wterms = 0;        // CTA-uniform bound of products per lane copy (W >= 2)
    int cur_hist = -1;
    double cur_wscale = 0.0;
    // integer weights: before n more j-points, flush if a lane copy of the
    // weight records could exceed WINT_LIMIT products (NT / wint_k threads
    // share a copy; each piece sum then stays below 2^16 x 2^16)
    auto wint_room = [&](int n) {
        if (W < 2) return;
        const unsigned long long add = (unsigned long long)(NT / p.wint_k) * RI * (unsigned)n;
        if (wterms + add > (W == 3 ? WINT_LIMIT / 2 : WINT_LIMIT)) {
            if (p.wfold) {
                fold_records(p, s_whist);
            } else {
                flush_hist<G>(p, s_hist, s_whist, cur_hist, cur_wscale);
                since_flush = 0;
            }
            wterms = 0;
        }
        wterms += add;
    };
    __syncthreads();   // CTA-wide: shared histograms are clear

    for (;;) {
        if (tid == 0) cs.blk = atomicAdd(p.work_counter, 1);   // the list holds only this shard's blocks
        gsync<G>();
        const int bidx = cs.blk;
        if (bidx >= nblocks) break;
        const Block B = p.blocks[bidx];
        const TaskDev &T = p.tasks[B.task];
        if (T.hist != cur_hist || (W >= 2 && T.wscale != cur_wscale)) {
            flush_hist<G>(p, s_hist, s_whist, cur_hist, cur_wscale);
            cur_hist = T.hist;
            cur_wscale = T.wscale;
            since_flush = 0;
            wterms = 0;
        }
        const size_t hbase = (size_t)T.hist * nbins;
        const unsigned task_bits = (unsigned)B.task << 5;
        const int ax = B.cell % nx, ay = (B.cell / nx) % ny, az = B.cell / (nx * ny);

        // thread t holds the block's points RI t .. RI t + RI - 1: a warp covers
        // 32 RI consecutive (sub-cell ordered, so spatially compact) points
        IPts<RI> I;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int loc = RI * tid + r;
            I.idx[r] = B.start + loc;
            I.xa[r] = I.ya[r] = I.za[r] = 0.f;
            I.w[r] = 0.0;
            I.wm[r] = 0u;
            I.wl[r] = I.pf[r] = 0.f;
            I.x[r] = I.y[r] = I.z[r] = -1.0e18f;  // unused lane: far from every j (and from the +1e18 pad slot)
            if (loc < B.count) {
                float4 q = T.gi.rel[I.idx[r]];
                I.x[r] = q.x; I.y[r] = q.y; I.z[r] = q.z;
                I.wm[r] = __float_as_uint(q.w);
                if (W == 3) {
                    I.pf[r] = __uint2float_rn(I.wm[r]);
                    I.wl[r] = T.gi.wlo ? T.gi.wlo[I.idx[r]] : 0.f;
                }
                if (LOS == LOS_MID || W == 1) {
                    double4_32a a = T.gi.xw[I.idx[r]];
                    I.xa[r] = (float)a.x; I.ya[r] = (float)a.y; I.za[r] = (float)a.z;
                    I.w[r] = a.w;
                }
            }
        }
        {   // the warp's i-box (empty box if the warp holds no point)
            float lx = INFINITY, ly = INFINITY, lz = INFINITY;
            float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
#pragma unroll
            for (int r = 0; r < RI; ++r)
                if (RI * tid + r < B.count) {
                    lx = fminf(lx, I.x[r]); hx = fmaxf(hx, I.x[r]);
                    ly = fminf(ly, I.y[r]); hy = fmaxf(hy, I.y[r]);
                    lz = fminf(lz, I.z[r]); hz = fmaxf(hz, I.z[r]);
                }
            lx = warp_minf(lx); ly = warp_minf(ly); lz = warp_minf(lz);
            hx = warp_maxf(hx); hy = warp_maxf(hy); hz = warp_maxf(hz);
            if ((tid & 31) == 0)
                s_ibox[tid >> 5] = GBox{make_float4(lx, ly, lz, 0.f), make_float4(hx, hy, hz, 0.f)};
        }
        const int ni_w = min(max(B.count - (tid >> 5) * 32 * RI, 0), 32 * RI);

        // ---- phase A (auto): pairs inside the block, j > i ------------------
        if (T.is_auto) {
            const int lenA = (B.count + 1) & ~1;    // even; the pad slot is far away
            for (int f = tid; f < lenA; f += NT) {
                if (f < B.count) {
                    int pj = B.start + f;
                    float4 q = T.gj.rel[pj];
                    s_tx[f] = q.x; s_ty[f] = q.y; s_tz[f] = q.z;
                    if (W == 1) s_tw[f] = T.gj.xw[pj].w;
                    if (W >= 2) s_twm[f] = __float_as_uint(q.w);
                    if (W == 3) s_twl[f] = T.gj.wlo ? T.gj.wlo[pj] : 0.f;
                } else {
                    s_tx[f] = s_ty[f] = s_tz[f] = 1.0e18f;
                    if (W == 1) s_tw[f] = 0.0;
                    if (W >= 2) s_twm[f] = 0u;
                    if (W == 3) s_twl[f] = 0.f;
                }
            }
            gsync<G>();
            wint_room(lenA);
            const int ngA = (lenA + JG - 1) / JG;    // all groups evaluated
            const unsigned maskA = ngA >= 32 ? 0xffffffffu : (1u << ngA) - 1u;
            pair_tile<MODE, LOS, W, RI, LIN, true>(p, smem_hist, Tile{s_tx, s_ty, s_tz, s_tw, s_twm, s_twl}, lenA,
                                                   maskA, I, bc, lc, r2cut, hist_sa, whist_sa, hk4, hbase, s_q,
                                                   &cs.qn, s_seg, 0, -1, 0, B.start, task_bits);
            if (tid == 0) cand_local += (unsigned long long)B.count * (B.count - 1) / 2;
            since_flush += (unsigned long long)B.count * B.count;
            gsync<G>();
        }

        // ---- phase B: j-segments, in chunks ---------------------------------
        // grid: the stencil rows, ROWCHUNK at a time; tree: the i-block's list
        // of (j-node, image) pairs, MAXSEG_T at a time
        // tree: virtual segment 0 of an auto count is the rest of the i-node
        // after this block (same node, no offset), then the listed nodes
        int ts0 = 0, tvirt = 0, trest = 0, node_end = 0;
        if constexpr (TREE) {
            ts0 = p.tseg_off[B.cell];
            if (T.is_auto) {
                const int2 r = p.tblk_j[B.cell];
                node_end = r.x + r.y;
                trest = (node_end > B.start + B.count) ? 1 : 0;
            }
            tvirt = p.tseg_off[B.cell + 1] - ts0 + trest;
        }
        const int nchunk = TREE ? (tvirt + MAXSEG_T - 1) / MAXSEG_T : (p.nrows + ROWCHUNK - 1) / ROWCHUNK;
        for (int ch = 0; ch < nchunk; ++ch) {
            if constexpr (TREE) {
                // segment k: a listed j-node's points, staged relative to the
                // i-node's centre through the offset of the two centres
                const int v0 = ch * MAXSEG_T;
                const int ns = min(MAXSEG_T, tvirt - v0);
                const double *ci = p.tcen_i + 3 * (size_t)B.cell;
                for (int k = tid; k < ns; k += NT) {
                    const int v = v0 + k;
                    if (v < trest) {
                        s_soff[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                        s_seg[k] = make_int4(B.start + B.count, node_end - B.start - B.count, k, 13);
                        continue;
                    }
                    const int2 e = p.tseg[ts0 + v - trest];
                    const int2 r = p.tblk_j[e.x];
                    const double *cj = p.tcen_j + 3 * (size_t)e.x;
                    const double sx = (double)(e.y / 9 - 1), sy = (double)((e.y / 3) % 3 - 1),
                                 sz = (double)(e.y % 3 - 1);
                    s_soff[k] = make_float4(
                        __double2float_rn(__dsub_rn(__dadd_rn(cj[0], __dmul_rn(sx, p.g.L[0])), ci[0])),
                        __double2float_rn(__dsub_rn(__dadd_rn(cj[1], __dmul_rn(sy, p.g.L[1])), ci[1])),
                        __double2float_rn(__dsub_rn(__dadd_rn(cj[2], __dmul_rn(sz, p.g.L[2])), ci[2])),
                        0.f);
                    s_seg[k] = make_int4(r.x, r.y, k, e.y);
                }
                if (tid == 0) cs.nseg = ns;
                gsync<G>();
            } else {
                const int r0 = ch * ROWCHUNK;
                const int r1 = min(r0 + ROWCHUNK, p.nrows);
                if (tid == 0) {
                    int ns = 0;
                    const int cell_end = T.gi.cell_start[B.cell + 1];
                    if (T.is_auto && r0 == 0 && cell_end > B.start + B.count) {
                        // rest of the own cell after this block (j > i for all)
                        s_seg[0] = make_int4(B.start + B.count, cell_end - B.start - B.count, 0, 13);
                        ns = 1;
                    }
                    cs.nseg = ns;
                }
                gsync<G>();
                build_segments(p, T.gj, ax, ay, az, r0, r1, s_seg, &cs.nseg);
                gsync<G>();
            }
            const int nseg = cs.nseg;
            gsync<G>();                 // every thread has read nseg before it changes
            if (nseg == 0) continue;
            const int total = seg_scan<G>(s_seg, nseg, s_tmp);
            // The chunk's j-points form ngt groups of JG; tile t holds the
            // groups t, t + ntiles, t + 2 ntiles, ...: every tile mixes all rows
            // of the chunk, so the warps (each pruning against its own i-box)
            // get similar work per tile.
            constexpr int GPT = TJ / JG;
            const int ngt = (total + JG - 1) / JG;
            const int ntiles = (ngt + GPT - 1) / GPT;
            auto tile_groups = [&](int t) { return (ngt - t + ntiles - 1) / ntiles; };
            if (tid == 0) cand_local += (unsigned long long)total * B.count;

            // staging registers (TJ / NT slots per thread)
            constexpr int SPT = TJ / NT;
            float4 rq[SPT];
            double rw[SPT];
            float rwl[SPT];
            int rcx[SPT], rmeta[SPT], rimg[SPT];
            bool rv[SPT];
            auto load_tile = [&](int t) {
#pragma unroll
                for (int s = 0; s < SPT; ++s) {
                    const int slot = tid + s * NT;
                    const int f = ((slot / JG) * ntiles + t) * JG + (slot % JG);
                    rv[s] = f < total && slot / JG < tile_groups(t);
                    if (rv[s]) {
                        int4 sg = s_seg[seg_find(s_seg, nseg, f)];
                        int pj = sg.x + (f - sg.y);
                        rq[s] = T.gj.rel[pj];
                        if constexpr (!TREE) rcx[s] = T.gj.cx[pj];
                        rmeta[s] = sg.z;
                        rimg[s] = sg.w;
                        if (W == 1) rw[s] = T.gj.xw[pj].w;
                        if (W == 3) rwl[s] = T.gj.wlo ? T.gj.wlo[pj] : 0.f;
                    }
                }
            };
            auto store_tile = [&](int t) {
                const int buf = t & 1;
                const int len = tile_groups(t) * JG;   // whole groups; missing points are pads
#pragma unroll
                for (int s = 0; s < SPT; ++s) {
                    const int slot = tid + s * NT;
                    float x = 1.0e18f, y = 1.0e18f, z = 1.0e18f;   // pad slot
                    double wv = 0.0;
                    if (rv[s]) {
                        if constexpr (TREE) {
                            const float4 o = s_soff[rmeta[s]];
                            x = o.x + rq[s].x;
                            y = o.y + rq[s].y;
                            z = o.z + rq[s].z;
                        } else {
                            int wrapx = rimg[s] / 9 - 1;
                            int dxc = rcx[s] - ax + wrapx * nx;
                            int dyc = (int)(short)(rmeta[s] & 0xFFFF);
                            int dzc = rmeta[s] >> 16;
                            x = fmaf((float)dxc, c32x, rq[s].x);
                            y = fmaf((float)dyc, c32y, rq[s].y);
                            z = fmaf((float)dzc, c32z, rq[s].z);
                        }
                        wv = rw[s];
                    }
                    if (slot < len) {
                        s_tx[buf * TJ + slot] = x;
                        s_ty[buf * TJ + slot] = y;
                        s_tz[buf * TJ + slot] = z;
                        if (W == 1) s_tw[buf * TJ + slot] = wv;
                        if (W >= 2) s_twm[buf * TJ + slot] = rv[s] ? __float_as_uint(rq[s].w) : 0u;
                        if (W == 3) s_twl[buf * TJ + slot] = rv[s] ? rwl[s] : 0.f;
                    }
                    // boxes of the j-groups (JG consecutive slots each)
                    const GBox gb = lane_group_box(x, y, z, rv[s]);
                    if ((tid & (JG - 1)) == 0) s_gbox[buf][slot / JG] = gb;
                }
            };

            load_tile(0);
            store_tile(0);
            gsync<G>();
            for (int t = 0; t < ntiles; ++t) {
                const int buf = t & 1;
                const int len = tile_groups(t) * JG;
                if (t + 1 < ntiles) load_tile(t + 1);
                wint_room(len);
                const unsigned gm = group_mask(s_gbox[buf], s_ibox[tid >> 5], len / JG, t, ntiles,
                                               total, ni_w, r2cut, &cs.pruned);
                pair_tile<MODE, LOS, W, RI, LIN, false>(
                    p, smem_hist,
                    Tile{s_tx + buf * TJ, s_ty + buf * TJ, s_tz + buf * TJ, s_tw + buf * TJ,
                         s_twm + buf * TJ, s_twl + buf * TJ},
                    len, gm, I, bc, lc, r2cut, hist_sa, whist_sa, hk4, hbase, s_q, &cs.qn, s_seg,
                    nseg, t, ntiles, B.start, task_bits);
                since_flush += (unsigned long long)len * B.count;
                if (t + 1 < ntiles) store_tile(t + 1);
                // one decision for the whole CTA, taken at the barrier: read
                // after it, the count could already include pushes of the next
                // tile by a faster warp, and the drain holds barriers itself
                if (gsync_or<G>(cs.qn >= LQ / 2))
                    drain_rescue<MODE, LOS, G>(p, s_q, cs, &s_base);
                if (since_flush > FLUSH_LIMIT / G) {
                    flush_hist<G>(p, s_hist, s_whist, cur_hist, cur_wscale);
                    since_flush = 0;
                    wterms = 0;
                }
            }
            gsync<G>();
        }
        drain_rescue<MODE, LOS, G>(p, s_q, cs, &s_base);
        gsync<G>();
    }
    drain_rescue<MODE, LOS, G>(p, s_q, cs, &s_base);
    flush_hist<G>(p, s_hist, s_whist, cur_hist, cur_wscale);
    if (tid == 0 && cand_local) atomicAdd(&p.counters[0], cand_local);
    if (tid == 0 && cs.pruned) atomicAdd(&p.counters[3], cs.pruned);
}

// ---------------------------------------------------------------------------
// plain FP64 kernel: the binary64 definition for every candidate pair
// ---------------------------------------------------------------------------
template <int MODE, int LOS, bool W>
__global__ void __launch_bounds__(NT) k_pairs_f64(const __grid_constant__ PairParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CtaShared cs;
    __shared__ int s_tmp[8];

    const SmemLayout Ly = smem_layout(p, true);
    double *s_Ea = (double *)(smem + Ly.ea);
    double *s_Eb = (double *)(smem + Ly.eb);
    int *s_hist = (int *)(smem + Ly.hist);
    double *s_whist = (double *)(smem + Ly.whist);
    int4 *s_seg = (int4 *)(smem + Ly.seg);
    double4_32a *s_tile = (double4_32a *)(smem + Ly.tile);
    int2 *s_meta = (int2 *)(smem + Ly.meta);

    const int tid = threadIdx.x;
    for (int k = tid; k <= p.n_a; k += NT) s_Ea[k] = p.Ea[k];
    for (int k = tid; k <= p.n_b; k += NT) s_Eb[k] = p.Eb[k];
    if (p.smem_hist_ok) {
        const int copies = (p.priv ? NT / 32 : 1) * p.hist_k;
        for (int k = tid; k < p.nbins_smem * copies; k += NT) s_hist[k] = 0;
        if (W) for (int k = tid; k < p.nbins_smem * p.hist_k; k += NT) s_whist[k] = 0.0;
    }
    const int K = p.hist_k, lane_copy = tid & (K - 1);
    int *my_hist = s_hist + (p.priv ? (tid >> 5) * p.nbins_smem * K : 0) + lane_copy;
    double *my_whist = s_whist + lane_copy;
    const int nx = p.g.ng[0], ny = p.g.ng[1];
    const int nblocks = *p.nblocks;
    unsigned long long cand_local = 0, since_flush = 0;
    int cur_hist = -1;
    __syncthreads();

    for (;;) {
        if (tid == 0) cs.blk = atomicAdd(p.work_counter, 1);   // the list holds only this shard's blocks
        __syncthreads();
        const int bidx = cs.blk;
        if (bidx >= nblocks) break;
        const Block B = p.blocks[bidx];
        const TaskDev &T = p.tasks[B.task];
        if (T.hist != cur_hist) {
            flush_hist(p, s_hist, s_whist, cur_hist);
            cur_hist = T.hist;
            since_flush = 0;
        }
        const size_t hbase = (size_t)T.hist * p.nbins;
        const int ax = B.cell % nx, ay = (B.cell / nx) % ny, az = B.cell / (nx * ny);
        const bool have_i = tid < B.count;   // FP64 path: one i-point per thread
        const int ii = B.start + tid;
        double4_32a a = have_i ? T.gi.xw[ii] : make_double4_32a(0, 0, 0, 0);

        auto add = [&](int bin, double wj) {
            if (p.smem_hist_ok) {
                atomicAdd(&my_hist[bin * K], 1);
                if (W) atomicAdd(&my_whist[bin * K], __dmul_rn(a.w, wj));
            } else {
                atomicAdd(&p.hist[hbase + bin], 1ull);
                if (W) atomicAdd(&p.whist[hbase + bin], __dmul_rn(a.w, wj));
            }
        };
        auto eval = [&](const double4_32a &b, int img) {
            int bin = f64_pair_bin<MODE, LOS>(a, b, img, p.g, s_Ea, p.n_a, s_Eb, p.n_b);
            if (bin >= 0) add(bin, b.w);
        };

        if (T.is_auto) {
            for (int f = tid; f < B.count; f += NT) {
                int pj = B.start + f;
                s_tile[f] = T.gj.xw[pj];
                s_meta[f] = make_int2(pj, 13);
            }
            __syncthreads();
            if (have_i)
                for (int jj = tid + 1; jj < B.count; ++jj) eval(s_tile[jj], 13);
            if (tid == 0) cand_local += (unsigned long long)B.count * (B.count - 1) / 2;
            since_flush += (unsigned long long)B.count * B.count;
            __syncthreads();
        }
        const int cell_end = T.gi.cell_start[B.cell + 1];
        for (int r0 = 0; r0 < p.nrows; r0 += ROWCHUNK) {
            const int r1 = min(r0 + ROWCHUNK, p.nrows);
            if (tid == 0) {
                int ns = 0;
                if (T.is_auto && r0 == 0 && cell_end > B.start + B.count) {
                    s_seg[0] = make_int4(B.start + B.count, cell_end - B.start - B.count, 0, 13);
                    ns = 1;
                }
                cs.nseg = ns;
            }
            __syncthreads();
            build_segments(p, T.gj, ax, ay, az, r0, r1, s_seg, &cs.nseg);
            __syncthreads();
            const int nseg = cs.nseg;
            __syncthreads();                 // every thread has read nseg before it changes
            if (nseg == 0) continue;
            const int total = seg_scan(s_seg, nseg, s_tmp);
            for (int t0 = 0; t0 < total; t0 += TJ64) {
                const int len = min(TJ64, total - t0);
                for (int f = tid; f < len; f += NT) {
                    int k = seg_find(s_seg, nseg, t0 + f);
                    int4 sg = s_seg[k];
                    int pj = sg.x + (t0 + f - sg.y);
                    s_tile[f] = T.gj.xw[pj];
                    s_meta[f] = make_int2(pj, sg.w);
                }
                __syncthreads();
                if (have_i)
                    for (int jj = 0; jj < len; ++jj) eval(s_tile[jj], s_meta[jj].y);
                if (tid == 0) cand_local += (unsigned long long)len * B.count;
                since_flush += (unsigned long long)len * B.count;
                __syncthreads();
                if (since_flush > FLUSH_LIMIT) {
                    flush_hist(p, s_hist, s_whist, cur_hist);
                    since_flush = 0;
                }
            }
        }
        __syncthreads();
    }
    flush_hist(p, s_hist, s_whist, cur_hist);
    if (tid == 0 && cand_local) atomicAdd(&p.counters[0], cand_local);
}

// ---------------------------------------------------------------------------
// rescue kernel: binary64 definition for every queued pair
// ---------------------------------------------------------------------------
template <int MODE, int LOS>
__global__ void __launch_bounds__(256) k_rescue(const __grid_constant__ PairParams p) {
    const unsigned long long n = min(*p.qcount, p.qcap);
    for (unsigned long long k = blockIdx.x * 256ull + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * 256ull) {
        uint3 e = p.queue[k];
        const int task = (int)(e.z >> 5), img = (int)(e.z & 31);
        const TaskDev &T = p.tasks[task];
        double4_32a a = T.gi.xw[e.x];
        double4_32a b = T.gj.xw[e.y];
        int bin = f64_pair_bin<MODE, LOS>(a, b, img, p.g, p.Ea, p.n_a, p.Eb, p.n_b);
        if (bin >= 0) {
            size_t h = (size_t)T.hist * p.nbins + bin;
            atomicAdd(&p.hist[h], 1ull);
            if (p.weighted) atomicAdd(&p.whist[h], __dmul_rn(a.w, b.w));
        }
    }
}

// ---------------------------------------------------------------------------
// instantiation helpers
// ---------------------------------------------------------------------------
template <int MODE, int LOS>
using PairKernel = void (*)(PairParams);

// Kernel variant for (weighted, i-points per thread, linear bins).  Linear
// bins are specialised only where they apply: s, and (s, mu) along z.
template <int MODE, int LOS>
PairKernel<MODE, LOS> pick_f32(const PairParams &p, int ipt) {
    constexpr bool LINOK = (MODE == MODE_S) || (MODE == MODE_SMU && LOS == LOS_Z) || MODE == MODE_SIGPI;
    const bool lin = LINOK && p.lin;
    if constexpr (LINOK) {
        // several thread groups per CTA (large histograms): floor bins, 2 i-points
        if (p.groups > 1 && lin && !p.wint)
            return p.weighted ? k_pairs_f32<MODE, LOS, 1, 2, true, 4> : k_pairs_f32<MODE, LOS, 0, 2, true, 4>;
    }
    if (p.weighted) {
        if constexpr (LINOK) {
            if (lin && p.wint && p.wcorr) return ipt == 4 ? k_pairs_f32<MODE, LOS, 3, 4, true>
                                                          : k_pairs_f32<MODE, LOS, 3, 2, true>;
            if (lin && p.wint) return ipt == 4 ? k_pairs_f32<MODE, LOS, 2, 4, true>
                                               : k_pairs_f32<MODE, LOS, 2, 2, true>;
        }
        if (ipt == 4) return lin ? k_pairs_f32<MODE, LOS, 1, 4, LINOK> : k_pairs_f32<MODE, LOS, 1, 4, false>;
        return lin ? k_pairs_f32<MODE, LOS, 1, 2, LINOK> : k_pairs_f32<MODE, LOS, 1, 2, false>;
    }
    if (ipt == 4) return lin ? k_pairs_f32<MODE, LOS, 0, 4, LINOK> : k_pairs_f32<MODE, LOS, 0, 4, false>;
    return lin ? k_pairs_f32<MODE, LOS, 0, 2, LINOK> : k_pairs_f32<MODE, LOS, 0, 2, false>;
}

// Tree variant (one thread group) for RI i-points per thread.
template <int MODE, int LOS, int RI>
PairKernel<MODE, LOS> pick_f32_tree_ri(const PairParams &p) {
    constexpr bool LINOK = (MODE == MODE_S) || (MODE == MODE_SMU && LOS == LOS_Z) || MODE == MODE_SIGPI;
    const bool lin = LINOK && p.lin;
    if (p.weighted) {
        if constexpr (LINOK) {
            if (lin && p.wint && p.wcorr) return k_pairs_f32<MODE, LOS, 3, RI, true, 1, true>;
            if (lin && p.wint) return k_pairs_f32<MODE, LOS, 2, RI, true, 1, true>;
        }
        return lin ? k_pairs_f32<MODE, LOS, 1, RI, LINOK, 1, true> : k_pairs_f32<MODE, LOS, 1, RI, false, 1, true>;
    }
    return lin ? k_pairs_f32<MODE, LOS, 0, RI, LINOK, 1, true> : k_pairs_f32<MODE, LOS, 0, RI, false, 1, true>;
}

template <int MODE, int LOS>
PairKernel<MODE, LOS> pick_f32_tree(const PairParams &p, int ipt) {
    return ipt == 4 ? pick_f32_tree_ri<MODE, LOS, 4>(p) : pick_f32_tree_ri<MODE, LOS, 2>(p);
}

template <int MODE, int LOS>
cudaError_t launch_kernel_f32(PairKernel<MODE, LOS> k, const PairParams &p, int grid, size_t smem,
                              cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, NT * p.groups, smem, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int MODE, int LOS>
int occupancy_kernel_f32(PairKernel<MODE, LOS> k, const PairParams &p, size_t smem) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT * p.groups, smem) != cudaSuccess) return 0;
    return nb;
}

template <int MODE, int LOS>
cudaError_t launch_mode_f32(const PairParams &p, int ipt, int grid, size_t smem, cudaStream_t st) {
    return launch_kernel_f32<MODE, LOS>(pick_f32<MODE, LOS>(p, ipt), p, grid, smem, st);
}

template <int MODE, int LOS>
int occupancy_mode_f32(const PairParams &p, int ipt, size_t smem) {
    return occupancy_kernel_f32<MODE, LOS>(pick_f32<MODE, LOS>(p, ipt), p, smem);
}

template <int MODE, int LOS>
cudaError_t launch_mode_f32_tree(const PairParams &p, int ipt, int grid, size_t smem,
                                 cudaStream_t st) {
    return launch_kernel_f32<MODE, LOS>(pick_f32_tree<MODE, LOS>(p, ipt), p, grid, smem, st);
}

template <int MODE, int LOS>
int occupancy_mode_f32_tree(const PairParams &p, int ipt, size_t smem) {
    return occupancy_kernel_f32<MODE, LOS>(pick_f32_tree<MODE, LOS>(p, ipt), p, smem);
}

template <int MODE, int LOS>
cudaError_t launch_mode_f64(const PairParams &p, int grid, size_t smem, cudaStream_t st) {
    void (*k)(PairParams) = p.weighted ? k_pairs_f64<MODE, LOS, true> : k_pairs_f64<MODE, LOS, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, NT, smem, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int MODE, int LOS>
int occupancy_mode_f64(const PairParams &p, size_t smem) {
    void (*k)(PairParams) = p.weighted ? k_pairs_f64<MODE, LOS, true> : k_pairs_f64<MODE, LOS, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
    return nb;
}

template <int MODE, int LOS>
cudaError_t launch_mode_rescue(const PairParams &p, int grid, cudaStream_t st) {
    k_rescue<MODE, LOS><<<grid, 256, 0, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pc
