// Known-answer source for the oracle's Philox4x32-10 on the GPU: cuRAND's
// device function curand_Philox4x32_10 (the generator of Salmon et al.,
// SC'11, as the CUDA toolkit ships it), called on given (counter, key) pairs.
// Test infrastructure only: built by the test that uses it.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void kat_philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    const uint4 r = curand_Philox4x32_10(c, k);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// d_ctr [n, 4], d_key [n, 2], d_out [n, 4]: device arrays on the current
// device.  Returns 0, or a cudaError_t of the launch or the synchronisation.
extern "C" int curand_philox4x32_10(const uint32_t *d_ctr, const uint32_t *d_key, uint32_t *d_out,
                                    int n) {
    if (n <= 0) return 0;
    kat_philox_kernel<<<(n + 255) / 256, 256>>>(d_ctr, d_key, d_out, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    return (int)cudaDeviceSynchronize();
}
