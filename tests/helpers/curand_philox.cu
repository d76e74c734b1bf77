// Test helper (not part of the library): cuRAND's device Philox4_32_10 for
// known-answer checks of the oracle's Philox. curand_init(seed, subseq,
// 4 * j) positions the counter at (lo j, hi j, lo subseq, hi subseq) with
// key (lo seed, hi seed); the first curand4 then returns Philox of that
// counter.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void curand_philox_kernel(const unsigned long long* seed, const unsigned long long* j,
                                     const unsigned long long* subseq, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed[i], subseq[i], 4ull * j[i], &st);
  out[i] = curand4(&st);
}

extern "C" int curand_philox(const unsigned long long* seed, const unsigned long long* j,
                             const unsigned long long* subseq, uint4* out, int n, void* stream) {
  if (n <= 0) return 0;
  curand_philox_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(seed, j, subseq, out, n);
  return (int)cudaGetLastError();
}
