// Prints the first draws of cuRAND's Philox4_32_10 generator for a few
// (seed, subsequence) pairs, one line per draw:
//   seed subsequence draw x y z w
// A state initialised with (seed, subsequence s, offset 0) returns, on draw
// n, Philox4x32-10 of the counter (n, 0, s_lo, s_hi) under the key
// (seed_lo, seed_hi); the test compares these lines with the oracle.
#include <cstdio>
#include <cstdint>
#include <curand_kernel.h>

__global__ void draws(const unsigned long long *seeds, const unsigned long long *subs, int n, int ndraw, uint4 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seeds[i], subs[i], 0ull, &st);
    for (int d = 0; d < ndraw; ++d) out[i * ndraw + d] = curand4(&st);
}

int main() {
    const unsigned long long seeds[] = {0ull, 1ull, 0x0123456789ABCDEFull, 0xFFFFFFFFFFFFFFFFull, 42ull, 0xDEADBEEF00000007ull};
    const unsigned long long subs[] = {0ull, 7ull, 1ull << 33, 0xFFFFFFFFull, 123456789ull, 0x8000000000000001ull};
    const int n = 6, ndraw = 3;
    unsigned long long *ds, *dq;
    uint4 *dout, hout[n * ndraw];
    cudaMalloc(&ds, sizeof(seeds));
    cudaMalloc(&dq, sizeof(subs));
    cudaMalloc(&dout, sizeof(hout));
    cudaMemcpy(ds, seeds, sizeof(seeds), cudaMemcpyHostToDevice);
    cudaMemcpy(dq, subs, sizeof(subs), cudaMemcpyHostToDevice);
    draws<<<1, 32>>>(ds, dq, n, ndraw, dout);
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    cudaMemcpy(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost);
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < ndraw; ++d) {
            const uint4 v = hout[i * ndraw + d];
            printf("%llu %llu %d %u %u %u %u\n", seeds[i], subs[i], d, v.x, v.y, v.z, v.w);
        }
    cudaFree(ds);
    cudaFree(dq);
    cudaFree(dout);
    return 0;
}
