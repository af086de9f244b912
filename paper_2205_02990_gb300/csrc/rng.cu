// Gaussian test matrices (Algorithm 2, first block): Philox4x32-10 + Box-Muller.
//
// Philox4x32 with 10 rounds follows its published definition (Salmon, Moraes, Dror, Shaw,
// SC'11): per round, counter words 0 and 2 are multiplied by 0xD2511F53 and 0xCD9E8D57; the
// new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85 between rounds. Each output gives two normals by the
// Box-Muller transform. The element layout is fixed by the public header (hbs_draw_gaussian).
// The kernel is a grid-stride loop over element pairs; it is bound by the FP64 transcendental
// throughput (log, sqrt, sincospi), not by the 16 bytes it writes per pair.
#include "hbs_internal.cuh"

namespace hbs {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// (top 52 bits of a*2^32 + b, plus 1/2) * 2^-52: exact, strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  const uint64_t word = (static_cast<uint64_t>(a) << 32) | b;
  return (static_cast<double>(word >> 12) + 0.5) * 0x1p-52;
}

__global__ void gaussian_kernel(int64_t count, uint32_t stream_id, uint32_t seed_lo,
                                uint32_t seed_hi, double* __restrict__ out) {
  const int64_t pairs = (count + 1) / 2;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < pairs;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 x = philox4x32_10(
        make_uint4(static_cast<uint32_t>(p), static_cast<uint32_t>(p >> 32), stream_id, 0u),
        make_uint2(seed_lo, seed_hi));
    const double u1 = uniform52(x.x, x.y);
    const double u2 = uniform52(x.z, x.w);
    const double rho = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[2 * p] = rho * cs;
    if (2 * p + 1 < count) out[2 * p + 1] = rho * sn;
  }
}

}  // namespace

cudaError_t launch_gaussian(int64_t count, uint32_t stream_id, uint64_t seed, double* out,
                            cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t pairs = (count + 1) / 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  int64_t blocks = (pairs + threads - 1) / threads;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 152) * 8;
  if (blocks > cap) blocks = cap;
  gaussian_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(
      count, stream_id, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), out);
  return cudaGetLastError();
}

}  // namespace hbs
