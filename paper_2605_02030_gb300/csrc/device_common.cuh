// Device helpers shared by the query kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "uhnsw.h"

namespace uhnsw_dev {

constexpr uint32_t kExpanded = 0x80000000u;  // beam entry already expanded
constexpr uint32_t kIdMask = 0x7fffffffu;
constexpr int32_t kEmpty = -1;
constexpr unsigned kFull = 0xffffffffu;

// (da, ia) before (db, ib) in the (distance, id) order used everywhere.
__device__ __forceinline__ bool pair_lt(float da, int32_t ia, float db, int32_t ib) {
  return da < db || (da == db && ia < ib);
}

// Row storage types: 16 bytes hold 4 FP32 or 8 FP16/BF16 values.
template <typename T> struct Elems16;
template <> struct Elems16<float> { static constexpr int n = 4; };
template <> struct Elems16<__half> { static constexpr int n = 8; };
template <> struct Elems16<__nv_bfloat16> { static constexpr int n = 8; };

__device__ __forceinline__ uint4 ldg16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

template <typename T>
__device__ __forceinline__ void unpack16(const uint4& v, float* out);

template <>
__device__ __forceinline__ void unpack16<float>(const uint4& v, float* out) {
  out[0] = __uint_as_float(v.x);
  out[1] = __uint_as_float(v.y);
  out[2] = __uint_as_float(v.z);
  out[3] = __uint_as_float(v.w);
}

template <>
__device__ __forceinline__ void unpack16<__half>(const uint4& v, float* out) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
    float2 f = __half22float2(h);
    out[2 * i] = f.x;
    out[2 * i + 1] = f.y;
  }
}

template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(const uint4& v, float* out) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
    float2 f = __bfloat1622float2(h);
    out[2 * i] = f.x;
    out[2 * i + 1] = f.y;
  }
}

// Hardware base-2 logarithm and exponential (the SFU instructions).
__device__ __forceinline__ float hw_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// |a|^p for the verification modes: general p as 2^(p log2 |a|) (two SFU
// operations; |0|^p = 2^-inf = 0), p = 0.5 and p = 1.5 through one square
// root (Section 2.1's fast cases), p = 1 and p = 2 without the SFU.
enum PMode { kPGeneral = 0, kPHalf = 1, kPThreeHalves = 2, kPOne = 3, kPTwo = 4 };

__device__ __forceinline__ int pmode_of(float p) {
  if (p == 1.0f) return kPOne;
  if (p == 2.0f) return kPTwo;
  if (p == 0.5f) return kPHalf;
  if (p == 1.5f) return kPThreeHalves;
  return kPGeneral;
}

template <int PM>
__device__ __forceinline__ float pow_term(float a, float p) {
  if (PM == kPOne) return a;
  if (PM == kPTwo) return a * a;
  if (PM == kPHalf) return hw_sqrt(a);
  if (PM == kPThreeHalves) return a * hw_sqrt(a);
  return hw_ex2(p * hw_lg2(a));
}

// Records the first error code of a launch into the sticky device word
// (err[0]; err[1..3] hold the site, value and limit of a failed index check).
__device__ __forceinline__ void set_error(int32_t* err, int32_t code) {
  if (err) atomicCAS(err, 0, code);
}

// Index check of the diagnostic build (compiled with -DUHNSW_CHECK): an index
// outside [0, limit) is recorded (code UHNSW_ECAPACITY, site, value, limit)
// and replaced by 0 so that the access stays inside the buffer.  In the
// normal build it is the identity.
__device__ __forceinline__ int64_t chk_idx(int64_t i, int64_t limit, int site, int32_t* err) {
#ifdef UHNSW_CHECK
  if (i < 0 || i >= limit) {
    if (err && atomicCAS(err, 0, UHNSW_ECAPACITY) == 0) {
      err[1] = site;
      err[2] = (int32_t)i;
      err[3] = (int32_t)limit;
    }
    return 0;
  }
#else
  (void)limit;
  (void)site;
  (void)err;
#endif
  return i;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t id, int bits) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - bits);
}

// Insert `id` into the open-addressing table (linear probing); true if it was
// absent.  The caller keeps the load at or below one half, so a free slot is
// always found within the table size.
__device__ __forceinline__ bool hash_insert(int32_t* tab, int bits, int32_t id, int32_t* err) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t s = hash_slot(id, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t old = atomicCAS(&tab[s], kEmpty, id);
    if (old == kEmpty) return true;
    if (old == id) return false;
    s = (s + 1u) & mask;
  }
  set_error(err, UHNSW_ECAPACITY);
  return false;
}

// Number of entries of the ascending (d, id) list [0, n) that precede (x, xi).
__device__ __forceinline__ int lower_bound_pair(const float* d, const uint32_t* id, int n, float x,
                                                int32_t xi) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (pair_lt(d[mid], (int32_t)(id[mid] & kIdMask), x, xi)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Block-wide merge of m unsorted new entries (nd, ni) into the ascending list
// (ld, li) of n entries, keeping the first `cap` of the union in (od, oi).
// Ids carry a flag in bit 31 that is preserved; flag-free ids are unique.
// sd/si is scratch for m entries.  Returns the new length; *first_flagless
// (if non-null) receives the smallest output position whose flag is clear
// (INT_MAX if none).  Must be called by every thread of the block; ends with
// a barrier.
__device__ __forceinline__ int block_merge(const float* ld, const uint32_t* li, int n,
                                           const float* nd, const uint32_t* ni, int m, float* sd,
                                           uint32_t* si, float* od, uint32_t* oi, int cap,
                                           int* first_flagless) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float x = nd[i];
    int32_t xi = (int32_t)(ni[i] & kIdMask);
    int r = 0;
    for (int j = 0; j < m; ++j) r += pair_lt(nd[j], (int32_t)(ni[j] & kIdMask), x, xi);
    r = (int)chk_idx(r, m, 8, nullptr);
    sd[r] = x;
    si[r] = ni[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int pos = lower_bound_pair(ld, li, n, sd[i], (int32_t)(si[i] & kIdMask)) + i;
    if (pos < cap) {
      od[pos] = sd[i];
      oi[pos] = si[i];
      if (first_flagless && !(si[i] & kExpanded)) atomicMin(first_flagless, pos);
    }
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int pos = lower_bound_pair(sd, si, m, ld[j], (int32_t)(li[j] & kIdMask)) + j;
    if (pos < cap) {
      od[pos] = ld[j];
      oi[pos] = li[j];
      if (first_flagless && !(li[j] & kExpanded)) atomicMin(first_flagless, pos);
    }
  }
  __syncthreads();
  int total = n + m;
  return total < cap ? total : cap;
}

// Two FP32 lanes in one 64-bit register: Blackwell's paired FP32 instructions
// (sub / add / fma .f32x2, IEEE round-to-nearest per element).
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f2_hsum(uint64_t v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return a + b;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

}  // namespace uhnsw_dev
