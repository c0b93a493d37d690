// Pair-separation histogram kernels (templates; instantiated per binning
// mode in pairs_*.cu).
//
// Work decomposition (grid traversal of Sect. 2.1 with the half-shell
// duplicate removal of Sect. 3.1): a persistent CTA repeatedly takes a block
// of up to NT * RI consecutive points of one cell (the i-points, kept in
// registers) and streams every candidate j-point of the neighbouring cells
// through shared memory.  Neighbours are visited row by row: for a stencil
// row (dy, dz) the cells (ax + xlo .. ax + xhi, ay + dy, az + dz) are
// contiguous in the cell-sorted arrays, so each row is one index range
// (split at most in three by periodic wrapping).  Periodic images are
// handled by shifting whole cells (Sect. 3.1), never by testing each pair.
//
// FP32 path: the j-point is staged as its offset from the i-cell centre,
// rel_j + delta * c, so a pair costs three subtractions and three
// multiply-adds.  The squared separation selects candidates; in-range pairs
// are binned through lookup tables over s, mu, sigma or pi (Sect. 3.2.3),
// each entry holding the single bin edge near that table cell.  A pair whose
// value lies within the proven FP32 error band of that edge is re-evaluated
// with the exact binary64 definition (queued for the rescue kernel), so the
// integer counts equal the binary64 definition exactly.
#pragma once

#include "pc_internal.cuh"

namespace pc {

constexpr unsigned long long FLUSH_LIMIT = 1ull << 30;

struct SmemLayout {
    size_t lut, ea, eb, hist, whist, seg, tile, meta, tw, q, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// FP32 path (f64 = false) and FP64 path (f64 = true) share one layout.
__host__ __device__ inline SmemLayout smem_layout(const PairParams &p, bool f64) {
    SmemLayout L;
    size_t o = 0;
    L.lut = o;
    o = align_up(o + (size_t)p.lut_total * sizeof(float2), 16);
    L.ea = o;
    o = align_up(o + (size_t)(p.n_a + 1) * sizeof(double), 16);
    L.eb = o;
    o = align_up(o + (size_t)(p.n_b + 1) * sizeof(double), 16);
    int copies = p.priv ? NT / 32 : 1;
    L.hist = o;
    if (p.smem_hist_ok) o = align_up(o + (size_t)p.nbins * copies * sizeof(int), 16);
    L.whist = o;
    if (p.smem_hist_ok && p.weighted) o = align_up(o + (size_t)p.nbins * sizeof(double), 16);
    L.seg = o;
    o = align_up(o + (size_t)MAXSEG * sizeof(int4), 16);
    int tj = f64 ? TJ64 : TJ;
    L.tile = o;
    o = align_up(o + (size_t)2 * tj * (f64 ? sizeof(double4_32a) : sizeof(float4)), 16);
    L.meta = o;
    o = align_up(o + (size_t)2 * tj * sizeof(int2), 16);
    L.tw = o;
    if (p.weighted && !f64) o = align_up(o + (size_t)2 * tj * sizeof(double), 16);
    L.q = o;
    o = align_up(o + (size_t)LQ * sizeof(uint3), 16);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// per-CTA state shared by both precisions
// ---------------------------------------------------------------------------
struct CtaShared {
    int blk;
    int nseg;
    int total;
    int qn;
};

// Exclusive prefix over the segment lengths held in seg[k].y (in place);
// returns the total.  All NT threads call it.
__device__ __forceinline__ int seg_scan(int4 *seg, int nseg, int *s_tmp) {
    // each thread owns a contiguous run of ceil(nseg / NT) segments
    const int tid = threadIdx.x;
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
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_tmp[w];
    int total = s_tmp[0] + s_tmp[1] + s_tmp[2] + s_tmp[3];
    int run = wbase + v - local;
    for (int k = b0; k < b1; ++k) {
        int len = seg[k].y;
        seg[k].y = run;
        run += len;
    }
    __syncthreads();
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
    for (int row = r0 + (int)threadIdx.x; row < r1; row += NT) {
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
template <int MODE, int LOS>
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
    atomicAdd(&p.counters[1], 1ull);
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

// Drain the CTA's staged rescue entries to the global queue (all threads).
template <int MODE, int LOS>
__device__ __forceinline__ void drain_rescue(const PairParams &p, uint3 *s_q, CtaShared &cs,
                                             unsigned long long *s_base) {
    int n = min(cs.qn, LQ);
    if (n == 0) return;
    if (threadIdx.x == 0) *s_base = atomicAdd(p.qcount, (unsigned long long)n);
    __syncthreads();
    unsigned long long base = *s_base;
    for (int k = threadIdx.x; k < n; k += NT) {
        unsigned long long g = base + k;
        if (g < p.qcap) p.queue[g] = s_q[k];
        else inline_rescue<MODE, LOS>(p, s_q[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) cs.qn = 0;
    __syncthreads();
}

// Add the CTA's shared histogram(s) into histogram `h` and clear them.
__device__ __forceinline__ void flush_hist(const PairParams &p, int *s_hist, double *s_whist,
                                           int h) {
    __syncthreads();
    if (p.smem_hist_ok && h >= 0) {
        const int copies = p.priv ? NT / 32 : 1;
        for (int b = threadIdx.x; b < p.nbins; b += NT) {
            long long v = 0;
            for (int c = 0; c < copies; ++c) {
                v += s_hist[c * p.nbins + b];
                s_hist[c * p.nbins + b] = 0;
            }
            if (v) atomicAdd(&p.hist[(size_t)h * p.nbins + b], (unsigned long long)v);
            if (p.weighted) {
                double w = s_whist[b];
                s_whist[b] = 0.0;
                if (w != 0.0) atomicAdd(&p.whist[(size_t)h * p.nbins + b], w);
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// FP32 binning of one in-range candidate
// ---------------------------------------------------------------------------
struct Bin32 {
    int bin;     // histogram index, valid only if ok
    bool ok;     // falls inside the histogram
    bool near;   // within an error band: needs the binary64 definition
};

__device__ __forceinline__ void lut_locate(const float2 *lut, const LutDesc &d, float v, int &k,
                                           float &edge) {
    // v >= 0 by construction; the unsigned clamp also sends any negative
    // index to the always-rescue sentinel cell
    int t = (int)min((unsigned)lut_index(v, d.inv_w), (unsigned)(d.T + 1));
    float2 e = lut[d.off + t];
    edge = e.x;
    k = __float_as_int(e.y) + (v >= e.x ? 1 : 0);
}

template <int MODE, int LOS>
__device__ __forceinline__ Bin32 bin_f32(const PairParams &p, const float2 *lut, float dx,
                                         float dy, float dz, float qxy, float s2, float ax_,
                                         float ay_, float az_) {
    Bin32 r;
    if (MODE == MODE_S) {
        float rs = rsqrtf(s2);
        float s = s2 * rs;
        int k; float e;
        lut_locate(lut, p.la, s, k, e);
        r.near = !(fabsf(s - e) >= p.eps_a);
        r.ok = (unsigned)k < (unsigned)p.n_a;
        r.bin = k;
        return r;
    }
    if (LOS == LOS_Z) {
        if (MODE == MODE_SMU) {
            float rs = rsqrtf(s2);
            float s = s2 * rs;
            float mu = fabsf(dz) * rs;
            int k, j; float e, em;
            lut_locate(lut, p.la, s, k, e);
            lut_locate(lut, p.lb, mu, j, em);
            float epsm = fmaf(p.mu_A, rs, p.mu_B);
            r.near = !(fabsf(s - e) >= p.eps_a) || !(fabsf(mu - em) >= epsm) || (epsm > p.mu_W);
            r.ok = (unsigned)k < (unsigned)p.n_a;
            r.bin = k * p.n_b + j;
            return r;
        }
        // (sigma, pi) along z
        float sg = qxy * rsqrtf(qxy);
        float pz = fabsf(dz);
        int k, j; float e, ep;
        lut_locate(lut, p.la, sg, k, e);
        lut_locate(lut, p.lb, pz, j, ep);
        r.near = !(fabsf(sg - e) >= p.eps_a) || !(fabsf(pz - ep) >= p.eps_b);
        r.ok = ((unsigned)k < (unsigned)p.n_a) && ((unsigned)j < (unsigned)p.n_b);
        r.bin = k * p.n_b + j;
        return r;
    }
    // midpoint line of sight: l = 2 x_i + d
    float lx = fmaf(2.0f, ax_, dx), ly = fmaf(2.0f, ay_, dy), lz = fmaf(2.0f, az_, dz);
    float sl = fmaf(dz, lz, fmaf(dy, ly, dx * lx));
    float ll = fmaf(lz, lz, fmaf(ly, ly, lx * lx));
    float rl = rsqrtf(ll);
    float pi = fabsf(sl) * rl;
    if (MODE == MODE_SMU) {
        float rs = rsqrtf(s2);
        float s = s2 * rs;
        float mu = pi * rs;
        int k, j; float e, em;
        lut_locate(lut, p.la, s, k, e);
        lut_locate(lut, p.lb, mu, j, em);
        float epsm = fmaf(p.mu_A, rs, p.mu_B);
        r.near = !(fabsf(s - e) >= p.eps_a) || !(fabsf(mu - em) >= epsm) || (epsm > p.mu_W);
        r.ok = (unsigned)k < (unsigned)p.n_a;
        r.bin = k * p.n_b + j;
        return r;
    }
    // sigma = |d x l| / |l|
    float cxp = fmaf(dy, lz, -dz * ly);
    float cyp = fmaf(dz, lx, -dx * lz);
    float czp = fmaf(dx, ly, -dy * lx);
    float cc = fmaf(czp, czp, fmaf(cyp, cyp, cxp * cxp));
    float sg = cc * rsqrtf(cc) * rl;
    int k, j; float e, ep;
    lut_locate(lut, p.la, sg, k, e);
    lut_locate(lut, p.lb, pi, j, ep);
    r.near = !(fabsf(sg - e) >= p.eps_a) || !(fabsf(pi - ep) >= p.eps_b);
    r.ok = ((unsigned)k < (unsigned)p.n_a) && ((unsigned)j < (unsigned)p.n_b);
    r.bin = k * p.n_b + j;
    return r;
}

// ---------------------------------------------------------------------------
// FP32 kernel
// ---------------------------------------------------------------------------
template <int MODE, int LOS, bool W, int RI>
__global__ void __launch_bounds__(NT) k_pairs_f32(const PairParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CtaShared cs;
    __shared__ int s_tmp[8];
    __shared__ unsigned long long s_base;

    const SmemLayout Ly = smem_layout(p, false);
    float2 *s_lut = (float2 *)(smem + Ly.lut);
    int *s_hist = (int *)(smem + Ly.hist);
    double *s_whist = (double *)(smem + Ly.whist);
    int4 *s_seg = (int4 *)(smem + Ly.seg);
    float4 *s_tile = (float4 *)(smem + Ly.tile);
    int2 *s_meta = (int2 *)(smem + Ly.meta);
    double *s_tw = (double *)(smem + Ly.tw);
    uint3 *s_q = (uint3 *)(smem + Ly.q);

    const int tid = threadIdx.x;
    for (int k = tid; k < p.lut_total; k += NT) s_lut[k] = p.lut[k];
    if (p.smem_hist_ok) {
        const int copies = p.priv ? NT / 32 : 1;
        for (int k = tid; k < p.nbins * copies; k += NT) s_hist[k] = 0;
        if (W) for (int k = tid; k < p.nbins; k += NT) s_whist[k] = 0.0;
    }
    if (tid == 0) cs.qn = 0;
    int *my_hist = s_hist + (p.priv ? (tid >> 5) * p.nbins : 0);

    const int nx = p.g.ng[0], ny = p.g.ng[1];
    const int nblocks = *p.nblocks;
    unsigned long long cand_local = 0;    // thread 0 only
    unsigned long long since_flush = 0;   // CTA-uniform
    int cur_hist = -1;
    __syncthreads();

    for (;;) {
        if (tid == 0) cs.blk = atomicAdd(p.work_counter, 1);
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

        // i-points in registers
        float xi[RI], yi[RI], zi[RI], xa[RI], ya[RI], za[RI];
        double wi[RI];
        int ii[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int loc = tid + r * NT;
            ii[r] = B.start + loc;
            xa[r] = ya[r] = za[r] = 0.f;
            wi[r] = 0.0;
            if (loc < B.count) {
                float4 q = T.gi.rel[ii[r]];
                xi[r] = q.x; yi[r] = q.y; zi[r] = q.z;
                if (LOS == LOS_MID || W) {
                    double4_32a a = T.gi.xw[ii[r]];
                    xa[r] = (float)a.x; ya[r] = (float)a.y; za[r] = (float)a.z;
                    wi[r] = a.w;
                }
            } else {
                xi[r] = yi[r] = zi[r] = 1.0e18f;   // never within range
            }
        }

        // one candidate pair (i-point r, staged j-point qj); the j metadata
        // is read only when the pair needs the binary64 definition
        auto count_pair = [&](int r, const float4 &qj, const int2 *mj, const double *wj) {
            float dx = qj.x - xi[r], dy = qj.y - yi[r], dz = qj.z - zi[r];
            float qxy = fmaf(dy, dy, dx * dx);
            float s2 = fmaf(dz, dz, qxy);
            if (s2 < p.r2cut) {
                Bin32 b = bin_f32<MODE, LOS>(p, s_lut, dx, dy, dz, qxy, s2, xa[r], ya[r], za[r]);
                if (!b.near) {
                    if (b.ok) {
                        if (p.smem_hist_ok) {
                            atomicAdd(&my_hist[b.bin], 1);
                            if (W) atomicAdd(&s_whist[b.bin], __dmul_rn(wi[r], *wj));
                        } else {
                            atomicAdd(&p.hist[hbase + b.bin], 1ull);
                            if (W) atomicAdd(&p.whist[hbase + b.bin], __dmul_rn(wi[r], *wj));
                        }
                    }
                } else {
                    int2 m = *mj;
                    push_rescue<MODE, LOS>(p, s_q, &cs.qn,
                                           make_uint3((unsigned)ii[r], (unsigned)m.x,
                                                      (unsigned)m.y | ((unsigned)B.task << 5)));
                }
            }
        };

        // ---- phase A (auto): pairs inside the block, j > i ------------------
        if (T.is_auto) {
            float4 *tb = s_tile;
            int2 *mb = s_meta;
            for (int f = tid; f < B.count; f += NT) {
                int pj = B.start + f;
                float4 q = T.gj.rel[pj];
                tb[f] = make_float4(q.x, q.y, q.z, 0.f);
                mb[f] = make_int2(pj, 13);
                if (W) s_tw[f] = T.gj.xw[pj].w;
            }
            __syncthreads();
            for (int jj = 0; jj < B.count; ++jj) {
                float4 qj = tb[jj];
                const int jidx = B.start + jj;
#pragma unroll
                for (int r = 0; r < RI; ++r)
                    if (jidx > ii[r]) count_pair(r, qj, mb + jj, s_tw + jj);
            }
            if (tid == 0) cand_local += (unsigned long long)B.count * (B.count - 1) / 2;
            since_flush += (unsigned long long)B.count * B.count;
            __syncthreads();
        }

        // ---- phase B: stencil rows, in chunks --------------------------------
        const int cell_end = T.gi.cell_start[B.cell + 1];
        for (int r0 = 0; r0 < p.nrows; r0 += ROWCHUNK) {
            const int r1 = min(r0 + ROWCHUNK, p.nrows);
            if (tid == 0) {
                int ns = 0;
                if (T.is_auto && r0 == 0 && cell_end > B.start + B.count) {
                    // rest of the own cell after this block (j > i for all)
                    s_seg[0] = make_int4(B.start + B.count, cell_end - B.start - B.count, 0, 13);
                    ns = 1;
                }
                cs.nseg = ns;
            }
            __syncthreads();
            build_segments(p, T.gj, ax, ay, az, r0, r1, s_seg, &cs.nseg);
            __syncthreads();
            const int nseg = cs.nseg;
            if (nseg == 0) continue;
            const int total = seg_scan(s_seg, nseg, s_tmp);
            const int ntiles = (total + TJ - 1) / TJ;

            // staging registers (TJ / NT slots per thread)
            constexpr int SPT = TJ / NT;
            float4 rq[SPT];
            int2 rm[SPT];
            double rw[SPT];
            int rcx[SPT], rmeta[SPT];
            auto load_tile = [&](int t) {
#pragma unroll
                for (int s = 0; s < SPT; ++s) {
                    int f = t * TJ + tid + s * NT;
                    rm[s].x = -1;
                    if (f < total) {
                        int k = seg_find(s_seg, nseg, f);
                        int4 sg = s_seg[k];
                        int pj = sg.x + (f - sg.y);
                        rq[s] = T.gj.rel[pj];
                        rcx[s] = T.gj.cx[pj];
                        rmeta[s] = sg.z;
                        rm[s] = make_int2(pj, sg.w);
                        if (W) rw[s] = T.gj.xw[pj].w;
                    }
                }
            };
            auto store_tile = [&](int buf) {
#pragma unroll
                for (int s = 0; s < SPT; ++s) {
                    if (rm[s].x < 0) continue;
                    int slot = tid + s * NT;
                    int wrapx = rm[s].y / 9 - 1;
                    int dxc = rcx[s] - ax + wrapx * nx;
                    int dyc = (int)(short)(rmeta[s] & 0xFFFF);
                    int dzc = rmeta[s] >> 16;
                    float4 v;
                    v.x = fmaf((float)dxc, p.g.c32[0], rq[s].x);
                    v.y = fmaf((float)dyc, p.g.c32[1], rq[s].y);
                    v.z = fmaf((float)dzc, p.g.c32[2], rq[s].z);
                    v.w = 0.f;
                    s_tile[buf * TJ + slot] = v;
                    s_meta[buf * TJ + slot] = rm[s];
                    if (W) s_tw[buf * TJ + slot] = rw[s];
                }
            };

            load_tile(0);
            store_tile(0);
            __syncthreads();
            for (int t = 0; t < ntiles; ++t) {
                const int buf = t & 1;
                const int len = min(TJ, total - t * TJ);
                if (t + 1 < ntiles) load_tile(t + 1);
                const float4 *tb = s_tile + buf * TJ;
                const int2 *mb = s_meta + buf * TJ;
                const double *wb = s_tw + buf * TJ;
#pragma unroll 2
                for (int jj = 0; jj < len; ++jj) {
                    float4 qj = tb[jj];
#pragma unroll
                    for (int r = 0; r < RI; ++r) count_pair(r, qj, mb + jj, wb + jj);
                }
                if (tid == 0) cand_local += (unsigned long long)len * B.count;
                since_flush += (unsigned long long)len * B.count;
                if (t + 1 < ntiles) store_tile(buf ^ 1);
                __syncthreads();
                if (cs.qn >= LQ / 2) drain_rescue<MODE, LOS>(p, s_q, cs, &s_base);
                if (since_flush > FLUSH_LIMIT) {
                    flush_hist(p, s_hist, s_whist, cur_hist);
                    since_flush = 0;
                }
            }
            __syncthreads();
        }
        drain_rescue<MODE, LOS>(p, s_q, cs, &s_base);
        __syncthreads();
    }
    drain_rescue<MODE, LOS>(p, s_q, cs, &s_base);
    flush_hist(p, s_hist, s_whist, cur_hist);
    if (tid == 0 && cand_local) atomicAdd(&p.counters[0], cand_local);
}

// ---------------------------------------------------------------------------
// plain FP64 kernel: the binary64 definition for every candidate pair
// ---------------------------------------------------------------------------
template <int MODE, int LOS, bool W>
__global__ void __launch_bounds__(NT) k_pairs_f64(const PairParams p) {
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
        const int copies = p.priv ? NT / 32 : 1;
        for (int k = tid; k < p.nbins * copies; k += NT) s_hist[k] = 0;
        if (W) for (int k = tid; k < p.nbins; k += NT) s_whist[k] = 0.0;
    }
    int *my_hist = s_hist + (p.priv ? (tid >> 5) * p.nbins : 0);
    const int nx = p.g.ng[0], ny = p.g.ng[1];
    const int nblocks = *p.nblocks;
    unsigned long long cand_local = 0, since_flush = 0;
    int cur_hist = -1;
    __syncthreads();

    for (;;) {
        if (tid == 0) cs.blk = atomicAdd(p.work_counter, 1);
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
                atomicAdd(&my_hist[bin], 1);
                if (W) atomicAdd(&s_whist[bin], __dmul_rn(a.w, wj));
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
__global__ void __launch_bounds__(256) k_rescue(const PairParams p) {
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
cudaError_t launch_mode_f32(const PairParams &p, int ipt, int grid, size_t smem, cudaStream_t st) {
    void (*k)(PairParams);
    if (p.weighted) k = (ipt == 2) ? k_pairs_f32<MODE, LOS, true, 2> : k_pairs_f32<MODE, LOS, true, 1>;
    else k = (ipt == 2) ? k_pairs_f32<MODE, LOS, false, 2> : k_pairs_f32<MODE, LOS, false, 1>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, NT, smem, st>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int MODE, int LOS>
int occupancy_mode_f32(const PairParams &p, int ipt, size_t smem) {
    void (*k)(PairParams);
    if (p.weighted) k = (ipt == 2) ? k_pairs_f32<MODE, LOS, true, 2> : k_pairs_f32<MODE, LOS, true, 1>;
    else k = (ipt == 2) ? k_pairs_f32<MODE, LOS, false, 2> : k_pairs_f32<MODE, LOS, false, 1>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
    return nb;
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
