// Measurement probes: the peak rates the kernels' roofline fractions are
// stated against, measured on the device at hand rather than assumed.
//   - SFU rate: base-2 logarithm and exponential, the two special-function
//     instructions of every general-p verification term (|d|^p as
//     2^(p log2 |d|)).
//   - Row-gather bandwidth: random rows of a given size read with 16-byte
//     vector loads, from a buffer that stays in L2 or one that does not.
// Neither probe is part of the query path.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "uhnsw_internal.h"

using namespace uhnsw_internal;

namespace uhnsw_dev {

// Eight independent chains per thread of x <- 2^(c log2 x): two SFU
// operations and one multiply per link.  With c < 1 and x > 0 the values
// stay normal and tend to 1.  The final test never holds for these inputs;
// it only keeps the chains alive.
__global__ void sfu_probe_kernel(float* sink, int iters, float c) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1.5f + 0.001f * (float)((threadIdx.x + 7 * j) & 63);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = hw_ex2(c * hw_lg2(x[j]));
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s < 0.f) sink[blockIdx.x] = s;
}

// A 32-bit integer mix (the finaliser of the MurmurHash3 family) used as a
// stateless random row index.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Each warp reads `per_warp` random rows of `row_chunks` 16-byte chunks; the
// lanes of a group of G = min(32, row_chunks) lanes share a row, and each
// group keeps four rows in flight.
__global__ void gather_probe_kernel(const uint4* __restrict__ buf, uint32_t rows, int row_chunks,
                                    int per_warp, unsigned* sink) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int G = row_chunks < 32 ? row_chunks : 32;
  const int groups = 32 / G;
  const int grp = lane / G, lg = lane - grp * G;
  unsigned acc = 0;
  if (grp < groups) {
    for (int i = grp * 4; i < per_warp; i += groups * 4) {
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t r = mix32(warp * 0x9E3779B1u + (uint32_t)(i + u)) % rows;
        const uint4* row = buf + (size_t)r * row_chunks;
        v[u] = make_uint4(0, 0, 0, 0);
        for (int c = lg; c < row_chunks; c += G) {
          const uint4 w = __ldg(row + c);
          v[u].x ^= w.x;
          v[u].y ^= w.y;
          v[u].z ^= w.z;
          v[u].w ^= w.w;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
  }
  if (acc == 0x9E3779B9u) sink[blockIdx.x & 1023] = acc;
}

}  // namespace uhnsw_dev

namespace {

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(UHNSW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Times `launch` on `st` with two events; returns the milliseconds in *ms.
template <typename F>
int timed(cudaStream_t st, F launch, float* ms, const char* what) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e == cudaSuccess ? UHNSW_OK : cuda_fail(e, what);
}

}  // namespace

extern "C" int uhnsw_probe_sfu(int32_t blocks_per_sm, int32_t iters, float* elapsed_ms,
                               double* ops, void* stream) {
  clear_error();
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !elapsed_ms || !ops)
    return fail(UHNSW_EINVAL, "uhnsw_probe_sfu: bad argument");
  const int sms = num_sms();
  if (sms < 1) return fail(UHNSW_ECUDA, "uhnsw_probe_sfu: no device");
  cudaStream_t st = (cudaStream_t)stream;
  float* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, (size_t)sms * blocks_per_sm * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_probe_sfu: sink");
  const int grid = sms * blocks_per_sm, block = 256;
  // one untimed launch first (module load, clocks)
  uhnsw_dev::sfu_probe_kernel<<<grid, block, 0, st>>>(sink, iters, 0.999f);
  int rc = timed(st, [&] { uhnsw_dev::sfu_probe_kernel<<<grid, block, 0, st>>>(sink, iters, 0.999f); },
                 elapsed_ms, "uhnsw_probe_sfu");
  cudaFree(sink);
  *ops = 2.0 * 8.0 * (double)iters * (double)grid * (double)block;
  return rc;
}

extern "C" int uhnsw_probe_gather(const void* buf, int64_t rows, int32_t row_bytes,
                                  int32_t per_warp, int32_t blocks_per_sm, float* elapsed_ms,
                                  double* bytes, void* stream) {
  clear_error();
  if (!buf || rows < 1 || rows > 0xffffffffll || row_bytes < 16 || (row_bytes & 15) ||
      per_warp < 128 || (per_warp & 127) || blocks_per_sm < 1 || blocks_per_sm > 64 || !elapsed_ms || !bytes ||
      (reinterpret_cast<uintptr_t>(buf) & 15))
    return fail(UHNSW_EINVAL, "uhnsw_probe_gather: bad argument");
  const int sms = num_sms();
  if (sms < 1) return fail(UHNSW_ECUDA, "uhnsw_probe_gather: no device");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 1024 * sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_probe_gather: sink");
  const int grid = sms * blocks_per_sm, block = 256;
  const int chunks = row_bytes / 16;
  const uint4* b = static_cast<const uint4*>(buf);
  uhnsw_dev::gather_probe_kernel<<<grid, block, 0, st>>>(b, (uint32_t)rows, chunks, per_warp, sink);
  int rc = timed(st, [&] {
    uhnsw_dev::gather_probe_kernel<<<grid, block, 0, st>>>(b, (uint32_t)rows, chunks, per_warp, sink);
  }, elapsed_ms, "uhnsw_probe_gather");
  cudaFree(sink);
  *bytes = (double)grid * (block / 32) * (double)per_warp * row_bytes;
  return rc;
}
