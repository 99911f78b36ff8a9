// Shared device helpers: Philox4x64-10, the device status word, launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpc_ring.h"

namespace mpc {

typedef unsigned long long u64;
typedef long long i64;

// ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------
// Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
//        c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key += (W0, W1) between rounds.
constexpr u64 kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr u64 kPhiloxM1 = 0xCA5A826395121157ull;
constexpr u64 kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr u64 kPhiloxW1 = 0xBB67AE8584CAA73Bull;

struct u64x4 {
  u64 v[4];
};

__device__ __forceinline__ u64x4 philox4x64_10(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0,
                                                u64 k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    // One full 64x64 -> 128-bit product per multiplier gives both halves.
    const unsigned __int128 p0 = (unsigned __int128)kPhiloxM0 * c0;
    const unsigned __int128 p1 = (unsigned __int128)kPhiloxM1 * c2;
    const u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0;
    const u64 hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;
    const u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  u64x4 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

__host__ __device__ __forceinline__ u64 stream_word2(unsigned role, unsigned sub, unsigned party) {
  return ((u64)role << 32) | ((u64)sub << 8) | (u64)party;
}

// Block `block` (4 words) of stream (seed, op_id, role, sub, party).
__device__ __forceinline__ u64x4 prg_block(u64 seed, u64 op_id, u64 word2, u64 block) {
  return philox4x64_10(block, op_id, word2, 0ull, seed, 0ull);
}

// ---- device status word ------------------------------------------------------
// Kernels record device-side failures in a per-device word (its address comes
// from device_status_ptr() on the host); mpc_sync_status() reads and clears it.
// The first failure wins.
__device__ __forceinline__ void record_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// ---- misc ----------------------------------------------------------------------
__host__ __device__ __forceinline__ i64 ceil_div(i64 a, i64 b) { return (a + b - 1) / b; }

__device__ __forceinline__ u64 sar(u64 v, int s) { return (u64)((i64)v >> s); }

// floor(s(v) / l) for l > 0.
__device__ __forceinline__ u64 floordiv_signed(u64 v, i64 l) {
  const i64 x = (i64)v;
  i64 q = x / l;
  if ((x % l != 0) && (x < 0)) q -= 1;
  return (u64)q;
}

// Four consecutive words starting at element i0 of an array of n words, with a
// ragged tail; 16-byte vector accesses when aligned.
struct Quad {
  u64 v[4];
};

// Plain (coherent) loads: outputs of some kernels may alias their inputs.
__device__ __forceinline__ Quad load4(const u64* a, i64 i0, i64 n) {
  Quad q;
  const u64* p = a + i0;
  if (i0 + 3 < n && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
    const ulonglong2 x = reinterpret_cast<const ulonglong2*>(p)[0];
    const ulonglong2 y = reinterpret_cast<const ulonglong2*>(p)[1];
    q.v[0] = x.x;
    q.v[1] = x.y;
    q.v[2] = y.x;
    q.v[3] = y.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) q.v[j] = (i0 + j < n) ? p[j] : 0ull;
  }
  return q;
}

__device__ __forceinline__ void store4(u64* a, i64 i0, i64 n, const Quad& q) {
  u64* p = a + i0;
  if (i0 + 3 < n && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
    reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(q.v[0], q.v[1]);
    reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(q.v[2], q.v[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i0 + j < n) p[j] = q.v[j];
  }
}

__device__ __forceinline__ Quad as_quad(const u64x4& b) {
  Quad q;
#pragma unroll
  for (int j = 0; j < 4; ++j) q.v[j] = b.v[j];
  return q;
}

inline unsigned grid_for(i64 work_items, int threads, i64 max_blocks = 148 * 32) {
  i64 b = ceil_div(work_items, threads);
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

}  // namespace mpc
