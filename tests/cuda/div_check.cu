// Test program: the solve body's reciprocal and division helpers against
// CUDA's IEEE reciprocal and quotient, bit for bit.
//   rcp_rn(b) == __frcp_rn(b) for every float b with exponent in [-100, 100];
//   div_from_rcp(a, b, rcp_rn(b)) == __fdiv_rn(a, b), and the zero-unsigned
//   variant too but for +0 in place of -0, on 2^30 pseudo-random pairs of
//   each of two domains: the sweep's (b a sum of two inverse masses in
//   [0.5, 2), |a| in [2^-40, 2^12), signed zeros among them) and the normals'
//   (b a distance in [2^-75, 2^2), |a| <= b).
// Prints one JSON line; exit status 0 iff no mismatch.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "acs_bodies.cuh"

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}
__device__ __forceinline__ float unit24(uint32_t h) { return (h >> 8) * (1.0f / 16777216.0f); }

__global__ void rcp_all(unsigned long long *bad) {
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < (1u << 23); m += gridDim.x * blockDim.x)
        for (int e = -100; e <= 100; ++e) {
            const float b = __uint_as_float(((uint32_t)(e + 127) << 23) | m);
            if (__float_as_uint(acs::rcp_rn(b)) != __float_as_uint(__frcp_rn(b))) atomicAdd(bad, 1ull);
        }
}

__global__ void div_pairs(int domain, uint64_t n, unsigned long long *bad) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t h1 = mix32((uint32_t)t * 2654435761u + 1u), h2 = mix32(h1 ^ 0x9e3779b9u), h3 = mix32(h2 + 0x85ebca6bu);
        float a, b;
        if (domain == 0) {
            b = __fadd_rn(0.5f + 1.5f * unit24(h1), 0.5f + 1.5f * unit24(h2));
            a = ldexpf(1.0f + unit24(h3), (int)(mix32(h3) % 52u) - 40);
            if ((h2 & 1023u) == 0u) a = 0.0f;      // a zero bias minus a zero speed
        } else {
            b = ldexpf(1.0f + unit24(h1), (int)(h2 % 77u) - 75);
            a = __fmul_rn(b, unit24(h3));
        }
        if (h3 & 1u) a = -a;
        const float q = __fdiv_rn(a, b), r = acs::rcp_rn(b);
        const float qz = acs::div_from_rcp_zero_unsigned(a, b, r);
        if (__float_as_uint(acs::div_from_rcp(a, b, r)) != __float_as_uint(q) ||
            __float_as_uint(qz) != __float_as_uint(q == 0.0f ? 0.0f : q))
            atomicAdd(bad, 1ull);
    }
}

int main() {
    unsigned long long *bad = nullptr, h[3] = {0, 0, 0};
    if (cudaMalloc(&bad, 3 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, 3 * sizeof(unsigned long long));
    rcp_all<<<148 * 8, 256>>>(bad);
    div_pairs<<<148 * 8, 256>>>(0, 1ull << 30, bad + 1);
    div_pairs<<<148 * 8, 256>>>(1, 1ull << 30, bad + 2);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost);
    printf("{\"rcp_values\": %llu, \"rcp_mismatches\": %llu, \"div_pairs\": %llu, \"div_mismatches_solve\": %llu, "
           "\"div_mismatches_normal\": %llu, \"cuda\": \"%s\"}\n",
           (unsigned long long)(1u << 23) * 201ull, h[0], 1ull << 30, h[1], h[2], cudaGetErrorString(e));
    return (e == cudaSuccess && !h[0] && !h[1] && !h[2]) ? 0 : 1;
}
