// Exhaustive error of the hardware base-2 logarithm (PTX lg2.approx.ftz.f32)
// over every positive normal binary32 input, against the binary64 log2.
// Prints the error model a + b |log2 x| that holds over all of them: a, the
// largest error where |log2 x| <= 1, and b, the largest error / |log2 x|
// elsewhere.  Used by tests/test_log2_bound.py to check the bound the
// log-bin bands assume.
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>

__global__ void k_lg2_err(unsigned first, unsigned count, unsigned long long *worst) {
    // worst[0]: max error with |log2 x| <= 1; worst[1]: max error / |log2 x|
    // beyond; each as (positive float bits << 32) | input bits
    unsigned long long best0 = 0, best1 = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x) {
        const unsigned b = first + i;
        const float x = __uint_as_float(b);
        float l;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
        const double ex = log2((double)x);
        const double e = fabs((double)l - ex);
        if (fabs(ex) <= 1.0) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint((float)e) << 32) | (unsigned long long)b;
            best0 = key > best0 ? key : best0;
        } else {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint((float)(e / fabs(ex))) << 32) |
                (unsigned long long)b;
            best1 = key > best1 ? key : best1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, best0, o);
        best0 = v > best0 ? v : best0;
        v = __shfl_xor_sync(0xffffffffu, best1, o);
        best1 = v > best1 ? v : best1;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&worst[0], best0);
        atomicMax(&worst[1], best1);
    }
}

int main() {
    unsigned long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return 1;
    cudaMemset(d, 0, sizeof(h));
    const unsigned first = 0x00800000u;              // smallest normal
    const unsigned count = 0x7F800000u - first;      // up to the largest finite
    k_lg2_err<<<152 * 16, 256>>>(first, count, d);
    if (cudaDeviceSynchronize() != cudaSuccess) return 2;
    cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    for (int k = 0; k < 2; ++k) {
        const unsigned eb = (unsigned)(h[k] >> 32), xb = (unsigned)h[k];
        float e, x;
        memcpy(&e, &eb, 4);
        memcpy(&x, &xb, 4);
        printf("%s %.9e at %.9e\n", k == 0 ? "a" : "b", (double)e, (double)x);
    }
    cudaFree(d);
    return 0;
}
