// Grid construction (Sect. 2.1: bounds, per-cell counts, grouping) and the
// i-block list that feeds the pair kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "pc_host.hpp"

namespace pc {

// ---------------------------------------------------------------------------
// periodic canonical form x - L floor(x / L), folded into [0, L)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double canon(double x, double L) {
    double y = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = __dsub_rn(y, L);
    return y;
}

// order-preserving map of a double onto a signed 64-bit key
__device__ __forceinline__ long long dkey(double v) {
    long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__host__ __device__ __forceinline__ double dunkey(long long k) {
    long long b = k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL);
    double v;
    memcpy(&v, &b, sizeof(v));
    return v;
}

// Bounds per axis and the smallest squared distance from the origin (the
// observer of the midpoint line of sight), as order-preserving keys:
// out[0..2] min, out[3..5] max, out[6] min of x^2 + y^2 + z^2 (rounded down
// so it never exceeds the exact value).
__global__ void k_aabb(const double *__restrict__ xyz, long long n, long long *out) {
    long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
    long long mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    long long r2min = LLONG_MAX;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = xyz[3 * i + a];
            long long k = dkey(x);
            mn[a] = min(mn[a], k);
            mx[a] = max(mx[a], k);
            r2 = __fma_rd(x, x, r2);
        }
        r2min = min(r2min, dkey(r2));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    for (int o = 16; o > 0; o >>= 1) r2min = min(r2min, __shfl_xor_sync(0xffffffffu, r2min, o));
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&out[a], mn[a]);
            atomicMax(&out[3 + a], mx[a]);
        }
        atomicMin(&out[6], r2min);
    }
}

pc_status aabb_device(const double *xyz, long long n, cudaStream_t st, double *lo, double *hi,
                      double *r2min) {
    long long init[7] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN,
                         LLONG_MAX};
    long long *d = nullptr;
    PC_CUDA(::pc::alloc_dev_async(&d, sizeof(init), st));
    PC_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, st));
    if (n > 0) {
        int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
        k_aabb<<<grid, 256, 0, st>>>(xyz, n, d);
        note_launch();
        PC_CUDA(cudaGetLastError());
    }
    long long res[7];
    PC_CUDA(cudaMemcpyAsync(res, d, sizeof(res), cudaMemcpyDeviceToHost, st));
    PC_CUDA(cudaFreeAsync(d, st));
    PC_CUDA(cudaStreamSynchronize(st));
    for (int a = 0; a < 3; ++a) {
        lo[a] = dunkey(res[a]);
        hi[a] = dunkey(res[3 + a]);
    }
    if (r2min) *r2min = n > 0 ? dunkey(res[6]) : 0.0;
    return PC_OK;
}

// ---------------------------------------------------------------------------
// cell ids and scatter
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_axis(double x, double lo, double c, int ng) {
    double f = floor(__ddiv_rn(__dsub_rn(x, lo), c));
    if (!(f >= 0.0)) return 0;
    if (f >= (double)(ng - 1)) return ng - 1;
    return (int)f;
}

// Sort key of a point: its cell, then (with sub_bits > 0) the Morton code of
// its sub-cell inside the cell, 2^sub_bits sub-cells per axis.  Points of one
// cell stay contiguous and neighbouring points end up close in memory, so a
// warp's consecutive points (and consecutive j-points) are spatially compact.
__device__ __forceinline__ unsigned morton3(unsigned x, unsigned y, unsigned z, int bits) {
    unsigned m = 0;
    for (int b = 0; b < bits; ++b)
        m |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) |
             (((z >> b) & 1u) << (3 * b + 2));
    return m;
}

__global__ void k_cell_ids(const double *__restrict__ xyz, int n, Geom g, int sub_bits,
                           int *__restrict__ cell, int *__restrict__ slot,
                           int *__restrict__ counts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int id[3];
    unsigned sub[3];
    const int S = 1 << sub_bits;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = xyz[3 * (size_t)i + a];
        if (g.periodic) x = canon(x, g.L[a]);
        id[a] = cell_axis(x, g.lo[a], g.c[a], g.ng[a]);
        double f = __ddiv_rn(__dsub_rn(__dsub_rn(x, g.lo[a]), __dmul_rn((double)id[a], g.c[a])), g.c[a]);
        int sa = (int)floor(f * S);
        sub[a] = (unsigned)min(max(sa, 0), S - 1);
    }
    int c = (id[2] * g.ng[1] + id[1]) * g.ng[0] + id[0];
    int key = (c << (3 * sub_bits)) | (int)morton3(sub[0], sub[1], sub[2], sub_bits);
    cell[i] = key;
    slot[i] = atomicAdd(&counts[key], 1);
}

// Cell starts from the starts of the sorted keys.
__global__ void k_cell_starts(const int *__restrict__ key_start, int ncell, int sub_bits,
                              int *__restrict__ cell_start) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    cell_start[c] = key_start[(size_t)c << (3 * sub_bits)];
}

// Weight statistics for the integer weight path, on each weight's binary32
// rounding hi: out[0] counts weights that are not finite, negative or whose
// hi is subnormal (or zero for a weight that is not), and binary64 weights
// that are not binary32 values and whose hi lies below 2^-78 (their
// remainder would lose bits to binary32 underflow); out[1] / out[2] receive
// the largest / smallest biased exponent of the non-zero his; out[3] counts
// the binary64 weights that are not binary32 values (remainder lo != 0).
__global__ void k_wstats(const void *__restrict__ w, int w_is_f32, int n, int *out) {
    int bad = 0, nlo = 0, emax = -1, emin = 1000;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float f;
        bool inexact = false;
        if (w_is_f32) {
            f = ((const float *)w)[i];
        } else {
            const double d = ((const double *)w)[i];
            f = __double2float_rn(d);
            inexact = (double)f != d;
        }
        const unsigned b = __float_as_uint(f);
        const int e = (int)((b >> 23) & 0xFF);
        if ((b >> 31) || e == 0xFF || (e == 0 && (b & 0x7FFFFF))) { ++bad; continue; }
        if (e == 0) {            // +0 (and -0 above counts as negative)
            if (inexact) ++bad;
            continue;
        }
        if (inexact) {
            if (e < 49) { ++bad; continue; }
            ++nlo;
        }
        emax = max(emax, e);
        emin = min(emin, e);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        nlo += __shfl_xor_sync(0xffffffffu, nlo, o);
        emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&out[0], bad);
        if (nlo) atomicAdd(&out[3], nlo);
        atomicMax(&out[1], emax);
        atomicMin(&out[2], emin);
    }
}

pc_status weight_stats(const void *w, int w_is_f32, int n, cudaStream_t st, int r[4]) {
    int init[4] = {0, -1, 1000, 0};
    int *ws = nullptr;
    cudaError_t e = ::pc::alloc_dev_async(&ws, sizeof(init), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n > 0) {
        int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
        k_wstats<<<blocks, 256, 0, st>>>(w, w_is_f32, n, ws);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, ws, sizeof(int) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ws) cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "weight statistics");
    return PC_OK;
}

// Packed integer weight (stored in the w lane of the FP32 point record): the
// binary32 significand M with its leading one (w = M 2^(e-150)), shifted up
// by 8 - (emax - e) (the grid's exponents span at most 8 binades), so that it
// fits 32 bits and a pair's exact 64-bit product is (M_i M_j) 2^(16 - k_i -
// k_j), k = emax - e.  Zero weights pack to 0.
__device__ __forceinline__ unsigned pack_weight(double wv, int emax, int span) {
    const unsigned b = __float_as_uint(__double2float_rn(wv));
    const int e = (int)((b >> 23) & 0xFF);
    if (e == 0) return 0u;
    return ((b & 0x7FFFFFu) | 0x800000u) << (span - (emax - e));
}

__global__ void k_scatter(const double *__restrict__ xyz, const void *__restrict__ w, int w_is_f32,
                          int wpack_emax, int wpack_span, int n, Geom g, int sub_bits,
                          const int *__restrict__ cell,
                          const int *__restrict__ slot, const int *__restrict__ key_start,
                          float4 *__restrict__ rel,
                          uint16_t *__restrict__ cxo, double4_32a *__restrict__ xw,
                          int *__restrict__ perm, float *__restrict__ wlo) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int key = cell[i];
    int pos = key_start[key] + slot[i];
    int c = key >> (3 * sub_bits);
    int id[3] = {c % g.ng[0], (c / g.ng[0]) % g.ng[1], c / (g.ng[0] * g.ng[1])};
    double x[3];
    float r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = xyz[3 * (size_t)i + a];
        if (g.periodic) v = canon(v, g.L[a]);
        x[a] = v;
        double o = __dadd_rn(g.lo[a], __dmul_rn((double)id[a] + 0.5, g.c[a]));
        r[a] = __double2float_rn(__dsub_rn(v, o));
    }
    double wv = 1.0;
    if (w) wv = w_is_f32 ? (double)((const float *)w)[i] : ((const double *)w)[i];
    const unsigned wp = (w && wpack_emax > 0) ? pack_weight(wv, wpack_emax, wpack_span) : 0u;
    rel[pos] = make_float4(r[0], r[1], r[2], __uint_as_float(wp));
    if (wlo) wlo[pos] = weight_lo(wv, wpack_emax);
    cxo[pos] = (uint16_t)id[0];
    xw[pos] = make_double4_32a(x[0], x[1], x[2], wv);
    perm[pos] = i;
}

// ---------------------------------------------------------------------------
// exclusive scan (three passes: per-tile scan, scan of tile totals, add)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_V = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int &total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int y = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        s_warp[lane] = y;   // inclusive warp totals
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    int base = warp ? s_warp[warp - 1] : 0;
    int r = base + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int *in, int *out, int n, int *tile_tot) {
    __shared__ int s_warp[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_V;
    int v[SCAN_V];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_excl_scan(sum, s_warp, total);
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_totals(int *tot, int ntiles, int *out, int n) {
    __shared__ int s_warp[32];
    int carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += SCAN_T) {
        int i = b0 + threadIdx.x;
        int v = (i < ntiles) ? tot[i] : 0;
        int total;
        int r = block_excl_scan(v, s_warp, total);
        if (i < ntiles) tot[i] = r + carry;
        carry += total;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_scan_add(int *out, int n, const int *tot) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tot[i / SCAN_TILE];
}

cudaError_t scan_exclusive(const int *in, int *out, int n, cudaStream_t st) {
    int ntiles = std::max(1, (n + SCAN_TILE - 1) / SCAN_TILE);
    int *tot = nullptr;
    cudaError_t e = ::pc::alloc_dev_async(&tot, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_scan_tiles<<<ntiles, SCAN_T, 0, st>>>(in, out, n, tot);
        note_launch();
    } else {
        cudaMemsetAsync(tot, 0, sizeof(int), st);
    }
    k_scan_totals<<<1, SCAN_T, 0, st>>>(tot, n > 0 ? ntiles : 1, out, n);
    note_launch();
    if (n > 0) {
        k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, n, tot);
        note_launch();
    }
    e = cudaGetLastError();
    cudaFreeAsync(tot, st);
    return e;
}

// Same scan with the tile-total buffer supplied by the caller (at least
// max(1, ceil(n / 4096)) ints); performs no allocation.
cudaError_t scan_exclusive_into(const int *in, int *out, int n, int *tot, cudaStream_t st) {
    int ntiles = std::max(1, (n + SCAN_TILE - 1) / SCAN_TILE);
    if (n > 0) {
        k_scan_tiles<<<ntiles, SCAN_T, 0, st>>>(in, out, n, tot);
        note_launch();
    } else {
        cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    k_scan_totals<<<1, SCAN_T, 0, st>>>(tot, n > 0 ? ntiles : 1, out, n);
    note_launch();
    if (n > 0) {
        k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, n, tot);
        note_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// block list
// ---------------------------------------------------------------------------
// Blocks per (task, cell): ceil(count / bi), or none for a cell outside the
// shard (cells whose index % shard_count != shard_index).
__global__ void k_block_counts(const TaskDev *tasks, int ntasks, int ncell, int bi, int shard_index,
                               int shard_count, int *cnt) {
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)ntasks * ncell) return;
    int t = (int)(gid / ncell), c = (int)(gid % ncell);
    const int *cs = tasks[t].gi.cell_start;
    int nc = cs[c + 1] - cs[c];
    cnt[gid] = (c % shard_count == shard_index) ? (nc + bi - 1) / bi : 0;
}

__global__ void k_block_emit(const TaskDev *tasks, int ntasks, int ncell, const int *off,
                             Block *blocks, int *nblocks) {
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)ntasks * ncell;
    if (gid == 0) *nblocks = off[tot];
    if (gid >= tot) return;
    int t = (int)(gid / ncell), c = (int)(gid % ncell);
    int o0 = off[gid], nb = off[gid + 1] - o0;
    if (nb == 0) return;
    const int *cs = tasks[t].gi.cell_start;
    int s = cs[c], nc = cs[c + 1] - s;
    for (int k = 0; k < nb; ++k) {
        int b0 = s + (int)((long long)k * nc / nb);
        int b1 = s + (int)((long long)(k + 1) * nc / nb);
        blocks[o0 + k] = Block{t, c, b0, b1 - b0};
    }
}

// Block list with every temporary supplied by the caller (tmp_tot: at least
// max(1, ceil((ntasks * ncell) / 4096)) ints); performs no allocation.
cudaError_t make_blocks_into(const TaskDev *tasks_dev, int ntasks, int ncell, int bi,
                             int shard_index, int shard_count, Block *blocks, int *nblocks_dev,
                             int *tmp_counts, int *tmp_offsets, int *tmp_tot, cudaStream_t st) {
    long long tot = (long long)ntasks * ncell;
    int g = (int)((tot + 255) / 256);
    if (shard_count < 1) shard_count = 1, shard_index = 0;
    if (g > 0) {
        k_block_counts<<<g, 256, 0, st>>>(tasks_dev, ntasks, ncell, bi, shard_index, shard_count,
                                          tmp_counts);
        note_launch();
    }
    cudaError_t e = scan_exclusive_into(tmp_counts, tmp_offsets, (int)tot, tmp_tot, st);
    if (e != cudaSuccess) return e;
    k_block_emit<<<std::max(g, 1), 256, 0, st>>>(tasks_dev, ntasks, ncell, tmp_offsets, blocks,
                                                 nblocks_dev);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pc

// ---------------------------------------------------------------------------
// public: grid build / free / info / aabb
// ---------------------------------------------------------------------------
using namespace pc;

extern "C" pc_status pc_aabb(const double *xyz, long long n, void *stream, double *lo,
                             double *hi) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!lo || !hi || n < 0 || (n > 0 && !xyz)) return fail(PC_EINVAL, "pc_aabb: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const double *dx = xyz;
    double *tmp = nullptr;
    if (n > 0 && !is_device_ptr(xyz)) {
        PC_CUDA(::pc::alloc_dev_async(&tmp, sizeof(double) * 3 * n, st));
        PC_CUDA(cudaMemcpyAsync(tmp, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        dx = tmp;
    }
    pc_status s = aabb_device(dx, n, st, lo, hi);
    if (tmp) cudaFreeAsync(tmp, st);
    cudaStreamSynchronize(st);
    return s;
}

static void grid_release(pc_grid *g) {
    if (!g) return;
    cudaFree(g->rel);
    cudaFree(g->cx);
    cudaFree(g->xw);
    cudaFree(g->cell_start);
    cudaFree(g->perm);
    cudaFree(g->wlo);
    delete g;
}

extern "C" void pc_free_grid(pc_grid *g) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (g) forget_grid(g);
    grid_release(g);
}

extern "C" pc_status pc_grid_info(const pc_grid *g, long long *n, double *cell_size) {
    if (!g) return fail(PC_EINVAL, "pc_grid_info: null grid");
    if (n) *n = g->n;
    if (cell_size) *cell_size = g->cell_size;
    return PC_OK;
}

extern "C" pc_status pc_build_grid(const double *xyz, const void *w, int w_is_f32, long long n,
                                   const pc_box *box, double r_max, const pc_opts *opt,
                                   void *stream, pc_grid **out) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (!out) return fail(PC_EINVAL, "pc_build_grid: out is NULL");
    *out = nullptr;
    if (!box) return fail(PC_EINVAL, "pc_build_grid: box is NULL");
    if (n < 0) return fail(PC_EINVAL, "pc_build_grid: n < 0");
    if (n > 0 && !xyz) return fail(PC_EINVAL, "pc_build_grid: xyz is NULL");
    if (n >= (1LL << 31) - 1) return fail(PC_EOVERFLOW, "pc_build_grid: n must be below 2^31");
    if (!(r_max > 0.0) || !isfinite(r_max))
        return fail(PC_EINVAL, "pc_build_grid: r_max must be positive and finite");
    pc_opts o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));

    // inputs on the device
    const double *dxyz = xyz;
    const void *dw = w;
    double *tmp_xyz = nullptr;
    void *tmp_w = nullptr;
    if (n > 0 && !is_device_ptr(xyz)) {
        PC_CUDA(::pc::alloc_dev_async(&tmp_xyz, sizeof(double) * 3 * n, st));
        PC_CUDA(cudaMemcpyAsync(tmp_xyz, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        dxyz = tmp_xyz;
    }
    size_t wbytes = (size_t)n * (w_is_f32 ? sizeof(float) : sizeof(double));
    if (w && n > 0 && !is_device_ptr(w)) {
        PC_CUDA(::pc::alloc_dev_async(&tmp_w, wbytes, st));
        PC_CUDA(cudaMemcpyAsync(tmp_w, w, wbytes, cudaMemcpyHostToDevice, st));
        dw = tmp_w;
    }
    auto cleanup = [&]() {
        if (tmp_xyz) cudaFreeAsync(tmp_xyz, st);
        if (tmp_w) cudaFreeAsync(tmp_w, st);
    };

    pc_grid *g = new pc_grid();
    memset(static_cast<void *>(g), 0, sizeof(*g));
    g->device = dev;
    g->n = (int)n;
    g->weighted = (w != nullptr);
    Geom &G = g->g;
    G.periodic = box->periodic ? 1 : 0;

    // bounds of the points
    double plo[3] = {0, 0, 0}, phi[3] = {0, 0, 0};
    if (G.periodic) {
        for (int a = 0; a < 3; ++a) {
            if (!(box->L[a] > 0.0) || !isfinite(box->L[a])) {
                cleanup();
                delete g;
                return fail(PC_EINVAL, "pc_build_grid: periodic box needs L > 0 on every axis");
            }
            if (!(r_max < 0.5 * box->L[a])) {
                cleanup();
                delete g;
                return fail(PC_EINVAL,
                            "pc_build_grid: r_max must stay below half the periodic box side");
            }
            G.L[a] = box->L[a];
            G.hL[a] = 0.5 * box->L[a];
            G.lo[a] = 0.0;
            plo[a] = 0.0;
            phi[a] = box->L[a];
        }
    } else {
        if (n > 0) {
            pc_status s = aabb_device(dxyz, n, st, plo, phi, &g->r2min);
            if (s != PC_OK) { cleanup(); delete g; return s; }
            for (int a = 0; a < 3; ++a)
                if (!isfinite(plo[a]) || !isfinite(phi[a])) {
                    cleanup();
                    delete g;
                    return fail(PC_EINVAL, "pc_build_grid: non-finite coordinates");
                }
        }
        bool given = box->hi[0] > box->lo[0] && box->hi[1] > box->lo[1] && box->hi[2] > box->lo[2];
        for (int a = 0; a < 3; ++a) {
            if (given) {
                if (n > 0 && (plo[a] < box->lo[a] || phi[a] > box->hi[a])) {
                    cleanup();
                    delete g;
                    return fail(PC_EINVAL, "pc_build_grid: points lie outside the given bounds");
                }
                G.lo[a] = box->lo[a];
            } else {
                G.lo[a] = plo[a];
            }
            G.L[a] = 0.0;
            G.hL[a] = 0.0;
        }
        if (given)
            for (int a = 0; a < 3; ++a) { plo[a] = box->lo[a]; phi[a] = box->hi[a]; }
    }
    for (int a = 0; a < 3; ++a) { g->pts_lo[a] = plo[a]; g->pts_hi[a] = phi[a]; }

    // cell geometry
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= std::max(phi[a] - plo[a], 1e-300);
    double c = o.cell_size > 0.0 ? o.cell_size : pc_suggest_cell_size(n, vol, r_max, 1);
    const long long MAXCELL = 1LL << 26;
    for (int iter = 0; iter < 200; ++iter) {
        long long tot = 1;
        for (int a = 0; a < 3; ++a) {
            double ext = phi[a] - plo[a];
            long long k;
            if (G.periodic) k = std::max(1LL, (long long)floor(ext / c));
            else k = std::max(1LL, (long long)ceil(ext / c));
            if (k > 65535) k = 65536;
            G.ng[a] = (int)k;
            tot *= k;
        }
        bool ok = tot <= MAXCELL && G.ng[0] <= 65535 && G.ng[1] <= 65535 && G.ng[2] <= 65535;
        if (ok) break;
        c *= 1.1;
    }
    if (G.periodic) {
        // neighbour offsets reach ceil(r / c) cells each way; a periodic axis
        // needs 2 * that + 1 distinct cells so no two offsets alias
        const double rr = r_max * (1.0 + 1e-4);
        for (int a = 0; a < 3; ++a) {
            while (G.ng[a] < 65535 &&
                   G.ng[a] < 2 * (long long)ceil(rr / (G.L[a] / G.ng[a])) + 1)
                G.ng[a] += 1;
        }
    }
    if ((long long)G.ng[0] * G.ng[1] * G.ng[2] > MAXCELL || G.ng[0] > 65535 ||
        G.ng[1] > 65535 || G.ng[2] > 65535) {
        cleanup();
        delete g;
        return fail(PC_EOVERFLOW, "pc_build_grid: too many cells for this box and separation");
    }
    g->cell_size = c;
    for (int a = 0; a < 3; ++a) {
        G.c[a] = G.periodic ? G.L[a] / G.ng[a] : c;
        G.c32[a] = (float)G.c[a];
    }
    g->ncell = G.ng[0] * G.ng[1] * G.ng[2];

    // weights usable by the integer weight path: every weight's binary32
    // rounding a non-negative normal value (or zero); exponent range recorded;
    // binary64 weights that are not binary32 values add their remainders
    g->wint = 0;
    if (dw && n > 0) {
        int res[4];
        pc_status ws = weight_stats(dw, w_is_f32, (int)n, st, res);
        if (ws != PC_OK) {
            cleanup();
            delete g;
            return ws;
        }
        // (the packed significands carry the exponent range: at most 8)
        if (res[0] == 0 && (res[1] < 0 || res[1] - res[2] <= WINT_GRID_SPAN)) {
            g->wint = 1;
            g->wemax = res[1] >= 0 ? res[1] : 1;      // all zero: any exponent works
            g->wemin = res[1] >= 0 ? res[2] : 1;
            g->wcorr = res[3] > 0 ? 1 : 0;
        }
    }

    // device arrays
    cudaError_t e = cudaSuccess;
    size_t nn = std::max<long long>(n, 1);
    e = ::pc::alloc_dev(&g->rel, sizeof(float4) * nn);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&g->cx, sizeof(uint16_t) * nn);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&g->xw, sizeof(double4_32a) * nn);
    if (e == cudaSuccess) e = ::pc::alloc_dev(&g->cell_start, sizeof(int) * (g->ncell + 1));
    if (e == cudaSuccess) e = ::pc::alloc_dev(&g->perm, sizeof(int) * nn);
    if (e == cudaSuccess && g->wcorr) e = ::pc::alloc_dev(&g->wlo, sizeof(float) * nn);
    if (e != cudaSuccess) {
        cleanup();
        grid_release(g);
        cudaGetLastError();
        return fail(PC_ENOMEM, "pc_build_grid: device allocation failed");
    }
    // sub-cell order inside cells: 8, 64 or 4096 Morton sub-cells when cells
    // hold enough points for them to matter (4096 on the 1500-point cells of
    // the tuned benchmark grid: 1 % fewer pairs past the group bounds than 64)
    const double per_cell = (double)n / g->ncell;
    int sub_bits = per_cell >= 1024.0 ? 4 : (per_cell >= 128.0 ? 2 : (per_cell >= 16.0 ? 1 : 0));
    while (sub_bits > 0 && ((long long)g->ncell << (3 * sub_bits)) > (1LL << 28)) --sub_bits;
    const int nkey = g->ncell << (3 * sub_bits);
    int *counts = nullptr, *cell = nullptr, *slot = nullptr, *key_start = nullptr;
    e = ::pc::alloc_dev_async(&counts, sizeof(int) * nkey, st);
    if (e == cudaSuccess) e = ::pc::alloc_dev_async(&key_start, sizeof(int) * ((size_t)nkey + 1), st);
    if (e == cudaSuccess) e = ::pc::alloc_dev_async(&cell, sizeof(int) * nn, st);
    if (e == cudaSuccess) e = ::pc::alloc_dev_async(&slot, sizeof(int) * nn, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int) * nkey, st);
    if (e == cudaSuccess && n > 0) {
        int blocks = (int)((n + 255) / 256);
        k_cell_ids<<<blocks, 256, 0, st>>>(dxyz, (int)n, G, sub_bits, cell, slot, counts);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_exclusive(counts, key_start, nkey, st);
    if (e == cudaSuccess) {
        k_cell_starts<<<(g->ncell + 1 + 255) / 256, 256, 0, st>>>(key_start, g->ncell, sub_bits,
                                                                  g->cell_start);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        int blocks = (int)((n + 255) / 256);
        k_scatter<<<blocks, 256, 0, st>>>(dxyz, dw, w_is_f32, g->wint ? g->wemax : 0,
                                          WINT_GRID_SPAN, (int)n, G,
                                          sub_bits, cell, slot, key_start, g->rel, g->cx, g->xw,
                                          g->perm, g->wlo);
        note_launch();
        e = cudaGetLastError();
    }
    if (key_start) cudaFreeAsync(key_start, st);
    if (counts) cudaFreeAsync(counts, st);
    if (cell) cudaFreeAsync(cell, st);
    if (slot) cudaFreeAsync(slot, st);
    cleanup();
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        grid_release(g);
        return cuda_fail(e, "pc_build_grid");
    }
    *out = g;
    return PC_OK;
}
