// Histogram-update micro-benchmark (Sect. 3.2.4): a stream of squared
// separations (drawn as in App. C) binned by one of the update algorithms of
// Sect. 3.2 -- binary search or reverse traversal over the squared edges
// (Sect. 3.2.1), index mapping for linear or logarithmic bins (Sect. 3.2.2),
// or the hybrid index lookup table of a given size (Sect. 3.2.3) -- into a
// shared-memory histogram.  Every method ends on the exact decision of the
// pair definition, bin k iff E_k <= s2 < E_{k+1} in binary64: the index
// mapping is corrected by comparisons with the neighbouring edges, and a
// table entry holds the range of bins its cell (widened by one cell each way
// for the rounding of the cell index) can reach, searched by reverse
// traversal.
//
// The samples are binary32, so every comparison runs in binary32 against the
// edges rounded up, U_k = the smallest binary32 value >= E_k: for a binary32
// v, v < E_k iff v < U_k (no binary32 value lies in [E_k, U_k) unless it is
// E_k itself).  The decisions are those of the binary64 definition while the
// kernel stays off GB300's narrow FP64 pipe.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_host.hpp"

namespace pc {

enum { HB_BSEARCH = 0, HB_REVERSE = 1, HB_MAP_LIN = 2, HB_MAP_LOG = 3, HB_LUT = 4 };

struct HistBenchParams {
    const float *s2;
    long long n;
    int repeat;
    int nb;            // bins
    int copies;        // lane copies of the shared histogram (power of 2)
    int T;             // table cells (HB_LUT)
    float f;           // table: cell = (int)(s2 f - c0), one rounding (FMA)
    float c0;
    float map_a, map_b;   // mapping: t = (g(s2) - map_a) * map_b, g = sqrt or log2
    const float *U;       // squared edges rounded up to binary32, nb + 1
    const unsigned *tab;  // table entries {lowest bin | highest bin << 16}
    unsigned long long *out;
};

// Bin of one binary32 sample, -1 outside [U_0, U_nb).
template <int M>
__device__ __forceinline__ int hist_bin(float v, const float *sE, const unsigned *stab,
                                        const HistBenchParams &p) {
    const int nb = p.nb;
    if (!(v >= sE[0] && v < sE[nb])) return -1;
    int k;
    if (M == HB_BSEARCH) {
        int lo = 0, hi = nb;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (v >= sE[mid]) lo = mid; else hi = mid;
        }
        k = lo;
    } else if (M == HB_REVERSE) {
        k = nb - 1;
        while (v < sE[k]) --k;
    } else if (M == HB_MAP_LIN || M == HB_MAP_LOG) {
        const float g = (M == HB_MAP_LIN) ? sqrtf(v) : log2f(v);
        const float t = (g - p.map_a) * p.map_b;
        k = (t > 0.f) ? (int)fminf(t, (float)(nb - 1)) : 0;
        while (k > 0 && v < sE[k]) --k;
        while (k + 1 < nb && v >= sE[k + 1]) ++k;
    } else {
        int c = (int)fmaf(v, p.f, -p.c0);
        c = min(max(c, 0), p.T - 1);
        const unsigned e = stab[c];
        const int lo = (int)(e & 0xFFFFu);
        k = (int)(e >> 16);
        while (k > lo && v < sE[k]) --k;
    }
    return k;
}

// VEC: the samples are 16-byte aligned and read four at a time (four
// independent bin searches per thread and load).
template <int M, bool VEC>
__global__ void __launch_bounds__(256) k_hist_s2(const __grid_constant__ HistBenchParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int nb = p.nb;
    float *sE = (float *)sm;
    unsigned *stab = (unsigned *)(sm + (((size_t)(nb + 1) * sizeof(float) + 15) & ~(size_t)15));
    int *shist = (int *)((unsigned char *)stab + (((size_t)(M == HB_LUT ? p.T : 0) * 4 + 15) & ~(size_t)15));
    for (int k = threadIdx.x; k <= nb; k += blockDim.x) sE[k] = p.U[k];
    if (M == HB_LUT)
        for (int k = threadIdx.x; k < p.T; k += blockDim.x) stab[k] = p.tab[k];
    for (int k = threadIdx.x; k < nb * p.copies; k += blockDim.x) shist[k] = 0;
    __syncthreads();
    const int cp = threadIdx.x & (p.copies - 1);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n4 = VEC ? p.n / 4 : 0;
    for (int rep = 0; rep < p.repeat; ++rep) {
        if (VEC) {
            const float4 *s4 = (const float4 *)p.s2;
            for (long long i = tid0; i < n4; i += stride) {
                const float4 q = s4[i];
                const int k0 = hist_bin<M>(q.x, sE, stab, p);
                const int k1 = hist_bin<M>(q.y, sE, stab, p);
                const int k2 = hist_bin<M>(q.z, sE, stab, p);
                const int k3 = hist_bin<M>(q.w, sE, stab, p);
                if (k0 >= 0) atomicAdd(&shist[k0 * p.copies + cp], 1);
                if (k1 >= 0) atomicAdd(&shist[k1 * p.copies + cp], 1);
                if (k2 >= 0) atomicAdd(&shist[k2 * p.copies + cp], 1);
                if (k3 >= 0) atomicAdd(&shist[k3 * p.copies + cp], 1);
            }
        }
        for (long long i = 4 * n4 + tid0; i < p.n; i += stride) {
            const int k = hist_bin<M>(p.s2[i], sE, stab, p);
            if (k >= 0) atomicAdd(&shist[k * p.copies + cp], 1);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        long long s = 0;
        for (int c = 0; c < p.copies; ++c) s += shist[k * p.copies + c];
        if (s) atomicAdd(&p.out[k], (unsigned long long)s);
    }
}

static int bin_of(const std::vector<double> &E, double v) {
    // largest k in [0, nb) with E[k] <= v (v clamped into the range first)
    const int nb = (int)E.size() - 1;
    int k = (int)(std::upper_bound(E.begin(), E.end(), v) - E.begin()) - 1;
    return std::min(std::max(k, 0), nb - 1);
}

}  // namespace pc

using namespace pc;

extern "C" pc_status pc_hist_s2(const float *s2, long long n, int repeat, const double *edges,
                                int nbins, int method, int table_size, void *stream,
                                long long *counts, float *ms) {
    std::lock_guard<std::mutex> lk(api_mutex());
    if (n < 0 || (n > 0 && !s2) || repeat < 1 || !edges || !counts)
        return fail(PC_EINVAL, "pc_hist_s2: bad arguments");
    if (nbins < 1 || nbins > 65535) return fail(PC_EINVAL, "pc_hist_s2: nbins must lie in [1, 65535]");
    for (int k = 0; k <= nbins; ++k)
        if (!(edges[k] >= 0.0) || !isfinite(edges[k]) || (k > 0 && !(edges[k] > edges[k - 1])))
            return fail(PC_EINVAL, "pc_hist_s2: edges must be finite, >= 0 and increasing");
    if (method < HB_BSEARCH || method > HB_LUT) return fail(PC_EINVAL, "pc_hist_s2: unknown method");
    if (method == HB_MAP_LOG && !(edges[0] > 0.0))
        return fail(PC_EINVAL, "pc_hist_s2: logarithmic mapping needs edges[0] > 0");
    if (method == HB_LUT && (table_size < 1 || table_size > 49152))
        return fail(PC_EINVAL, "pc_hist_s2: table_size must lie in [1, 49152]");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    PC_CUDA(cudaGetDevice(&dev));
    PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    HistBenchParams p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.repeat = repeat;
    p.nb = nbins;
    int copies = 32;
    while (copies > 1 && (size_t)nbins * copies * 4 > 16384) copies >>= 1;
    p.copies = copies;
    std::vector<double> E(nbins + 1);
    std::vector<float> U(nbins + 1);
    for (int k = 0; k <= nbins; ++k) {
        E[k] = edges[k] * edges[k];
        float u = (float)E[k];
        if ((double)u < E[k]) u = nextafterf(u, INFINITY);
        U[k] = u;
    }
    std::vector<unsigned> tab;
    if (method == HB_MAP_LIN) {
        p.map_a = (float)edges[0];
        p.map_b = (float)(nbins / (edges[nbins] - edges[0]));
    } else if (method == HB_MAP_LOG) {
        p.map_a = (float)log2(E[0]);
        p.map_b = (float)(nbins / (log2(E[nbins]) - log2(E[0])));
    } else if (method == HB_LUT) {
        // cells of the rescaled squared separation (Sect. 3.2.3, Eq. hist_ntable)
        const double f = (double)(table_size - 1) / std::max(E[nbins] - E[0], 1e-300);
        p.f = (float)f;
        const double fd = (double)p.f;
        const double c0 = floor(E[0] * fd);
        if (!(c0 < 16777216.0))
            return fail(PC_EUNSUPPORTED,
                        "pc_hist_s2: e[0]^2 f must stay below 2^24 (f = (table_size - 1) / "
                        "(e[n]^2 - e[0]^2)) for an exact binary32 cell offset");
        p.c0 = (float)c0;
        // table_size - 1 cells span the range at scale f; the last cell and
        // the clamp absorb the rounding of f and of the cell index
        p.T = table_size;
        tab.resize(table_size);
        for (int c = 0; c < table_size; ++c) {
            // the FMA rounds s2 f - c0 once (relative error 2^-24 on a value
            // below table_size), so a sample in cell c has exactly s2 f in
            // [c0 + c - 1, c0 + c + 1); bounds widened for their own rounding
            const double lo = std::max(E[0], (c0 + c - 1) / fd * (1.0 - 1e-12));
            const double hi = std::min(E[nbins], (c0 + c + 2) / fd * (1.0 + 1e-12));
            const int klo = bin_of(E, lo);
            const int khi = (c == table_size - 1) ? nbins - 1 : bin_of(E, hi);
            tab[c] = (unsigned)klo | ((unsigned)std::max(klo, khi) << 16);
        }
    }
    const size_t smem = (((size_t)(nbins + 1) * 4 + 15) & ~(size_t)15) +
                        (((size_t)(method == HB_LUT ? p.T : 0) * 4 + 15) & ~(size_t)15) +
                        (size_t)nbins * copies * 4;
    int optin = 0;
    PC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin) return fail(PC_EUNSUPPORTED, "pc_hist_s2: table and histogram exceed shared memory");

    void (*kern)(HistBenchParams) = nullptr;
    auto pick = [&](bool v4) -> void (*)(HistBenchParams) {
        switch (method) {
            case HB_BSEARCH: return v4 ? k_hist_s2<HB_BSEARCH, true> : k_hist_s2<HB_BSEARCH, false>;
            case HB_REVERSE: return v4 ? k_hist_s2<HB_REVERSE, true> : k_hist_s2<HB_REVERSE, false>;
            case HB_MAP_LIN: return v4 ? k_hist_s2<HB_MAP_LIN, true> : k_hist_s2<HB_MAP_LIN, false>;
            case HB_MAP_LOG: return v4 ? k_hist_s2<HB_MAP_LOG, true> : k_hist_s2<HB_MAP_LOG, false>;
            default: return v4 ? k_hist_s2<HB_LUT, true> : k_hist_s2<HB_LUT, false>;
        }
    };
    // the four-wide loads need a 16-byte aligned device address; a host
    // input is staged in a fresh (aligned) allocation
    const bool aligned = !is_device_ptr(s2) || (((uintptr_t)s2 & 15u) == 0);
    kern = pick(aligned);
    PC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
    if (per_sm < 1) return fail(PC_EUNSUPPORTED, "pc_hist_s2: kernel cannot be resident");
    const long long want = std::max(1LL, (n + 255) / 256);
    const int grid = (int)std::min<long long>((long long)sms * per_sm, want);
    // shared counts are 32-bit: one CTA handles at most ceil(n / grid) samples per repeat
    if ((double)((n + grid - 1) / grid) * repeat >= 2147483647.0)
        return fail(PC_EOVERFLOW, "pc_hist_s2: too many samples per CTA for 32-bit shared counts");

    const float *ds2 = s2;
    float *tmp = nullptr;
    unsigned long long *dout = nullptr;
    float *dE = nullptr;
    unsigned *dtab = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pc_status status = PC_OK;
    cudaError_t e = cudaSuccess;
    if (n > 0 && !is_device_ptr(s2)) {
        e = ::pc::alloc_dev_async(&tmp, sizeof(float) * n, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, s2, sizeof(float) * n, cudaMemcpyHostToDevice, st);
        ds2 = tmp;
    }
    if (e == cudaSuccess) e = ::pc::alloc_dev_async(&dout, sizeof(unsigned long long) * nbins, st);
    if (e == cudaSuccess) e = ::pc::alloc_dev_async(&dE, sizeof(float) * (nbins + 1), st);
    if (e == cudaSuccess && !tab.empty()) e = ::pc::alloc_dev_async(&dtab, sizeof(unsigned) * tab.size(), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, sizeof(unsigned long long) * nbins, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dE, U.data(), sizeof(float) * (nbins + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && dtab)
        e = cudaMemcpyAsync(dtab, tab.data(), sizeof(unsigned) * tab.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        p.s2 = ds2;
        p.U = dE;
        p.tab = dtab;
        p.out = dout;
        cudaEventRecord(e0, st);
        if (n > 0) {
            kern<<<grid, 256, smem, st>>>(p);
            note_launch();
        }
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        cudaMemcpyKind kd = is_device_ptr(counts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        e = cudaMemcpyAsync(counts, dout, sizeof(long long) * nbins, kd, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ms) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
    }
    if (e != cudaSuccess) status = cuda_fail(e, "pc_hist_s2");
    if (tmp) cudaFreeAsync(tmp, st);
    if (dout) cudaFreeAsync(dout, st);
    if (dE) cudaFreeAsync(dE, st);
    if (dtab) cudaFreeAsync(dtab, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    return status;
}
