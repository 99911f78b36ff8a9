// Limb-split ring GEMM on tcgen05 tensor cores (sm_103a).
//
// §5.3 of the paper splits 64-bit ring elements into 16-bit limbs and runs
// float64 GEMMs per limb pair.  On B300 the integer MMA (kind::i8) is not
// available for sm_103a, and float64 tensor throughput is tiny, so this engine
// keeps the idea but maps it to the bf16 tensor cores:
//
//  * every u64 operand word v is cut into 8 balanced base-256 digits
//    d_i in [-128, 127] with v = sum_i d_i 2^(8i) (mod 2^64); each digit is an
//    exact bf16 (a "plane" holds one digit index of a whole matrix);
//  * Z = sum_{i+j<8} 2^(8(i+j)) A_i B_j (mod 2^64): only the 36 digit pairs
//    with i + j < 8 can reach the low 64 bits;
//  * pairs with the same shift s = i + j share one fp32 TMEM accumulator
//    (8 accumulators of 128 x 64 fill all 512 TMEM columns);
//  * |d_i d_j| <= 2^14 and at most 8 pairs share a shift, so 128 K-steps keep
//    every partial sum within 2^24 where fp32 holds integers exactly.  Each
//    accumulator is therefore drained every 8 sub-steps of K = 16 (chunks
//    staggered by shift, so one drain overlaps the MMAs of the other seven)
//    into a 64-bit integer register sum R += int(acc_s) << 8s;
//  * the epilogue adds C, applies the optional truncation and stores.
//
// Operands arrive as planes written by limb_planes_{a,b}: A as [8][M][Kp]
// and B transposed as [8][N][Kp] (both K-major), with K-concatenated operand
// pairs (Z = C + A1 B1 + A2 B2 is one GEMM over [A1 | A2] and [B1 ; B2]).
//
// Warp roles (416 threads): warp 0 issues TMA loads (one thread); warps 1-4
// each issue the MMAs of two shifts, {w, 7 - w}, 9 per K sub-step (one thread
// per warp: a single issuing thread cannot keep the tensor pipe busy with
// N = 64 MMAs); warp 1 also allocates TMEM; warps 5-12 drain TMEM, two per
// lane quadrant (warp w reads lanes 32 (w % 4) .. +31), 32 columns each, and
// write the output.  Every wait is
// bounded: on a timeout the CTA records MPC_ETIMEOUT, waits (bounded) for its
// own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <string.h>

#include <mutex>

#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int BM = 128, BN = 64, KS = 16, STAGES = 4, NSHIFT = 8, CHUNK = 8;
constexpr int A_PLANE_BYTES = BM * KS * 2;             // 4 KiB
constexpr int B_PLANE_BYTES = BN * KS * 2;             // 2 KiB
constexpr int A_STAGE_BYTES = NSHIFT * A_PLANE_BYTES;  // 32 KiB
constexpr int B_STAGE_BYTES = NSHIFT * B_PLANE_BYTES;  // 16 KiB
constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int kIssuers = 4;      // MMA-issuing warps (1..4)
constexpr int kDrainWarps = 8;   // TMEM drain / epilogue warps (5..12)
constexpr int kThreads = 32 * (1 + kIssuers + kDrainWarps);
constexpr uint32_t TMEM_COLS = 512;
// Instruction descriptor, kind::f16: D f32 (bit 4), A bf16 (bits 7-9 = 1),
// B bf16 (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

struct LimbParams {
  CUtensorMap tmA[MPC_MAX_PARTIES];
  CUtensorMap tmB[MPC_MAX_PARTIES];
  const u64* C[MPC_MAX_PARTIES];
  u64* Z[MPC_MAX_PARTIES];
  u64* partial;  // split-K partial sums [splits][njobs][M][N] (splits > 1)
  i64 M, N, hw_out;
  int T;  // K sub-steps of 16
  int trunc_bits;
  int splits, njobs;
  int* status;
};

// ---- PTX wrappers ------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (and raises the CTA's abort flag) when the limit passes or another role
// already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

// Shared-memory matrix descriptor: K-major, 32-byte swizzle, rows of 32 bytes,
// 8-row groups 256 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
  d |= (uint64_t)(256 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                    // version
  d |= (uint64_t)6 << 61;                    // SWIZZLE_32B
  return d;
}

#define TMEM_LD_X32(taddr, r)                                                                  \
  asm volatile(                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "  \
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "  \
      "%28, %29, %30, %31}, [%32];"                                                             \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),    \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),             \
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),          \
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),          \
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),          \
        "=r"(r[31])                                                                            \
      : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The s + 1 digit-pair MMAs of shift S: D += sum_{i <= S} A_i B_{S - i}.
template <int S>
__device__ __forceinline__ void issue_shift_t(uint32_t d, uint64_t a0, uint64_t b0, bool start) {
  tc_mma(d, a0, b0 + (uint64_t)(S * (B_PLANE_BYTES >> 4)), start ? 0u : 1u);
#pragma unroll
  for (int i = 1; i <= S; ++i)
    tc_mma(d, a0 + (uint64_t)(i * (A_PLANE_BYTES >> 4)),
           b0 + (uint64_t)((S - i) * (B_PLANE_BYTES >> 4)), 1u);
}

// Shift s's chunk ends after sub-step t when t = s - 1 (mod CHUNK), or at the
// end t_end - 1 of the CTA's K range.
__device__ __forceinline__ bool chunk_ends(int t, int s, int t_end) {
  return (t % CHUNK) == ((s + CHUNK - 1) % CHUNK) || t == t_end - 1;
}

// The two shifts owned by MMA-issuer warp w: {w, 7 - w}, 9 digit-pair MMAs
// per K sub-step for every issuer.
template <int W>
__device__ __forceinline__ void issuer_loop(const LimbParams& p, uint32_t sbase, uint32_t tmem,
                                            int t_begin, int t_end, uint64_t* full_bar,
                                            uint64_t* empty_bar, uint64_t* accf_bar,
                                            uint64_t* acce_bar, volatile int* abort_flag) {
  constexpr int S0 = W, S1 = NSHIFT - 1 - W;
  uint32_t chunks0 = 0, chunks1 = 0;
  for (int t = t_begin; t < t_end; ++t) {
    const int st = (t - t_begin) % STAGES;
    const uint32_t ph = (uint32_t)((t - t_begin) / STAGES) & 1u;
    if (!mbar_wait(&full_bar[st], ph, abort_flag)) return;
    tc_fence_after();
    const uint64_t a0 = smem_desc_sw32(sbase + st * STAGE_BYTES);
    const uint64_t b0 = smem_desc_sw32(sbase + st * STAGE_BYTES + A_STAGE_BYTES);
    // A chunk of shift s starts right after one ended (or at t = t_begin).
    const bool start0 = (t == t_begin) || ((t - 1) % CHUNK) == ((S0 + CHUNK - 1) % CHUNK);
    const bool start1 = (t == t_begin) || ((t - 1) % CHUNK) == ((S1 + CHUNK - 1) % CHUNK);
    if (start0 && t > t_begin) {
      if (!mbar_wait(&acce_bar[S0], (chunks0 - 1u) & 1u, abort_flag)) return;
      tc_fence_after();
    }
    issue_shift_t<S0>(tmem + (uint32_t)(S0 * BN), a0, b0, start0);
    if (chunk_ends(t, S0, t_end)) {
      tc_commit(&accf_bar[S0]);
      chunks0++;
    }
    if (start1 && t > t_begin) {
      if (!mbar_wait(&acce_bar[S1], (chunks1 - 1u) & 1u, abort_flag)) return;
      tc_fence_after();
    }
    issue_shift_t<S1>(tmem + (uint32_t)(S1 * BN), a0, b0, start1);
    if (chunk_ends(t, S1, t_end)) {
      tc_commit(&accf_bar[S1]);
      chunks1++;
    }
    tc_commit(&empty_bar[st]);
  }
}

__global__ void __launch_bounds__(kThreads, 1) limb_gemm_kernel(const __grid_constant__ LimbParams p) {
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[NSHIFT], acce_bar[NSHIFT], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int job = blockIdx.z / p.splits, split = blockIdx.z % p.splits;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // This CTA's K sub-steps [t_begin, t_end).
  const int t_begin = (int)((i64)p.T * split / p.splits);
  const int t_end = (int)((i64)p.T * (split + 1) / p.splits);
  const uint32_t sbase = (smem_u32(dsmem) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], kIssuers);
    }
    for (int i = 0; i < NSHIFT; ++i) {
      mbar_init(&accf_bar[i], 1);
      mbar_init(&acce_bar[i], kDrainWarps);
    }
    mbar_init(&done_bar, kIssuers);
    // A timeout recorded by an earlier CTA (and not yet cleared by
    // mpc_sync_status) makes every later CTA skip its work and exit at once.
    abort_flag = (*(volatile int*)p.status == MPC_ETIMEOUT) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.tmA[job])));
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.tmB[job])));
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      int last_t[STAGES];
      for (int i = 0; i < STAGES; ++i) last_t[i] = -1;
      for (int t = t_begin; t < t_end; ++t) {
        const int st = (t - t_begin) % STAGES;
        const uint32_t ph = (uint32_t)((t - t_begin) / STAGES) & 1u;
        if (!mbar_wait(&empty_bar[st], ph ^ 1u, &abort_flag)) break;
        mbar_arrive_expect_tx(&full_bar[st], STAGE_BYTES);
        const uint32_t a_dst = sbase + st * STAGE_BYTES;
        tma_load_3d(a_dst, &p.tmA[job], &full_bar[st], t * KS, m0, 0);
        tma_load_3d(a_dst + A_STAGE_BYTES, &p.tmB[job], &full_bar[st], t * KS, n0, 0);
        last_t[st] = t - t_begin;
      }
      // Copies in flight must land before the CTA can leave (bounded).
      for (int i = 0; i < STAGES; ++i) {
        if (last_t[i] < 0) continue;
        const uint32_t ph = (uint32_t)(last_t[i] / STAGES) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full_bar[i], ph) && globaltimer() - t0 < kWaitLimitNs) {
        }
      }
    }
  } else if (warp <= kIssuers) {
    if (lane == 0) {
      // ---- MMA issuers: warp 1 + w owns shifts {w, 7 - w} ----
      switch (warp - 1) {
        case 0: issuer_loop<0>(p, sbase, tmem, t_begin, t_end, full_bar, empty_bar, accf_bar,
                               acce_bar, &abort_flag); break;
        case 1: issuer_loop<1>(p, sbase, tmem, t_begin, t_end, full_bar, empty_bar, accf_bar,
                               acce_bar, &abort_flag); break;
        case 2: issuer_loop<2>(p, sbase, tmem, t_begin, t_end, full_bar, empty_bar, accf_bar,
                               acce_bar, &abort_flag); break;
        default: issuer_loop<3>(p, sbase, tmem, t_begin, t_end, full_bar, empty_bar, accf_bar,
                                acce_bar, &abort_flag); break;
      }
      // All of this issuer's MMAs must finish before TMEM is released (bounded).
      tc_commit(&done_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&done_bar, 0) && globaltimer() - t0 < kWaitLimitNs) {
      }
    }
  } else {
    // ---- TMEM drain + epilogue: 8 warps, two per TMEM lane quadrant ----
    const int ew = warp - 1 - kIssuers;           // 0..7
    const int q = warp & 3;                       // lane quadrant this warp may access
    const int half = ew >> 2;                     // which 32 of the 64 columns
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 32);
    u64 R[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) R[j] = 0;
    uint32_t chunks[NSHIFT];
#pragma unroll
    for (int s = 0; s < NSHIFT; ++s) chunks[s] = 0;
    bool ok = true;
    for (int t = t_begin; t < t_end && ok; ++t) {
      for (int s = 0; s < NSHIFT; ++s) {
        if (!chunk_ends(t, s, t_end)) continue;
        if (!mbar_wait(&accf_bar[s], chunks[s] & 1u, &abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t v[32];
        TMEM_LD_X32(lane_base + (uint32_t)(s * BN), v);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[s]);
        chunks[s]++;
        const int sh = 8 * s;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int iv = __float2int_rz(__uint_as_float(v[j]));
          R[j] += (u64)(i64)iv << sh;
        }
      }
    }
    const i64 row = (i64)m0 + q * 32 + lane;
    const int c0 = n0 + half * 32;
    if (ok && !abort_flag && row < p.M) {
      if (p.splits > 1) {
        u64* part = p.partial + ((i64)split * p.njobs + job) * p.M * p.N + row * p.N;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if ((i64)c0 + j < p.N) part[c0 + j] = R[j];
      } else {
        const u64* C = p.C[job];
        u64* Z = p.Z[job];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const i64 col = (i64)c0 + j;
          if (col < p.N) {
            const i64 idx = gemm_out_index(row, col, p.M, p.N, p.hw_out);
            u64 v = R[j];
            if (C) v += C[idx];
            if (p.trunc_bits > 0) v = sar(v, p.trunc_bits);
            Z[idx] = v;
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) record_status(p.status, MPC_ETIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---- plane pre-pass ---------------------------------------------------------------------
// Balanced base-256 digits of v: v = sum_i d_i 2^(8i) mod 2^64, d_i in [-128, 127].
__device__ __forceinline__ void balanced_digits(u64 v, int d[8]) {
  int carry = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int t = (int)((v >> (8 * i)) & 255ull) + carry;
    carry = t >= 128;
    d[i] = t - (carry << 8);
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(int lo, int hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn((float)lo), b = __float2bfloat16_rn((float)hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Writes 8 consecutive k' of one row into the 8 planes of `out` ([8][rows][Kp]).
__device__ __forceinline__ void write_planes(const u64 v[8], __nv_bfloat16* out, i64 rows,
                                             i64 row, i64 Kp, i64 k0) {
  int d[8][8];  // [element][digit]
#pragma unroll
  for (int e = 0; e < 8; ++e) balanced_digits(v[e], d[e]);
#pragma unroll
  for (int pl = 0; pl < 8; ++pl) {
    uint4 w;
    w.x = pack_bf16x2(d[0][pl], d[1][pl]);
    w.y = pack_bf16x2(d[2][pl], d[3][pl]);
    w.z = pack_bf16x2(d[4][pl], d[5][pl]);
    w.w = pack_bf16x2(d[6][pl], d[7][pl]);
    *reinterpret_cast<uint4*>(out + ((i64)pl * rows + row) * Kp + k0) = w;
  }
}

struct PlaneJob {
  const u64* X1;  // first pair operand
  const u64* X2;  // second pair operand (or null)
  __nv_bfloat16* out;
};

// A side: X is [M][K] row-major; element (m, k') of [X1 | X2].
__global__ void __launch_bounds__(256) limb_planes_a(PlaneJob j0,
                                                      PlaneJob j1, PlaneJob j2, PlaneJob j3,
                                                      PlaneJob j4, PlaneJob j5, PlaneJob j6,
                                                      PlaneJob j7, i64 M, i64 K, i64 Kp) {
  const PlaneJob js[8] = {j0, j1, j2, j3, j4, j5, j6, j7};
  const PlaneJob& jb = js[blockIdx.y];
  const i64 kc = Kp / 8;
  const i64 total = M * kc;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const i64 m = i / kc, k0 = (i % kc) * 8;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const i64 k = k0 + e;
      v[e] = k < K ? jb.X1[m * K + k] : (jb.X2 && k < 2 * K) ? jb.X2[m * K + (k - K)] : 0ull;
    }
    write_planes(v, jb.out, M, m, Kp, k0);
  }
}

// B side: X is [K][N] row-major; planes are written transposed, [8][N][Kp].
// One CTA per tile of 64 k' x 32 n: coalesced row reads of X, digits into a
// shared-memory tile [plane][n][k'] (33-word rows: the transposed stores hit
// distinct banks), then each warp writes 128-byte runs of one plane row.
constexpr int PB_TK = 64, PB_TN = 32, PB_ROW = PB_TK / 2 + 1;  // words per smem row

__global__ void __launch_bounds__(256) limb_planes_b(PlaneJob j0,
                                                      PlaneJob j1, PlaneJob j2, PlaneJob j3,
                                                      PlaneJob j4, PlaneJob j5, PlaneJob j6,
                                                      PlaneJob j7, i64 N, i64 K, i64 Kp) {
  __shared__ uint32_t tile[8][PB_TN][PB_ROW];
  const PlaneJob js[8] = {j0, j1, j2, j3, j4, j5, j6, j7};
  const PlaneJob& jb = js[blockIdx.z];
  const i64 k0 = (i64)blockIdx.x * PB_TK, n0 = (i64)blockIdx.y * PB_TN;
  const int tid = threadIdx.x, nl = tid & 31, kq = tid >> 5;  // kq: 0..7
  const i64 n = n0 + nl;
  // Load + digit phase: thread (nl, kq) owns k' pairs 2 (kq + 8 j), j = 0..3.
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int kl = 2 * (kq + 8 * j);
    u64 v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const i64 k = k0 + kl + e;
      v[e] = 0;
      if (n < N) {
        if (k < K) v[e] = jb.X1[k * N + n];
        else if (jb.X2 && k < 2 * K) v[e] = jb.X2[(k - K) * N + n];
      }
    }
    int d0[8], d1[8];
    balanced_digits(v[0], d0);
    balanced_digits(v[1], d1);
#pragma unroll
    for (int pl = 0; pl < 8; ++pl) tile[pl][nl][kl >> 1] = pack_bf16x2(d0[pl], d1[pl]);
  }
  __syncthreads();
  // Store phase: 8 planes x 32 rows; each warp writes whole 128-byte row runs.
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < 8 * PB_TN; r += 8) {
    const int pl = r / PB_TN, row = r % PB_TN;
    const i64 nn = n0 + row;
    const i64 kk = k0 + 2 * lane;
    if (nn < N && kk < Kp)
      *reinterpret_cast<uint32_t*>(jb.out + ((i64)pl * N + nn) * Kp + kk) = tile[pl][row][lane];
  }
}

// B side of a convolution, gathered straight from the data (implicit im2col):
// the same tiling and stores as limb_planes_b, with element (k', n) read at its
// data position instead of from a materialised im2col matrix.  The CTA's 64 k'
// are decoded once into a shared tap table (offset ci h w + r w + s, r, s and
// the source pair); column n = (b, oh, ow) is decoded once per thread, so an
// element costs two bounds checks and an add.
__global__ void __launch_bounds__(256) limb_planes_b_conv(const ConvGather cg, int job,
                                                           __nv_bfloat16* out, i64 N, i64 K,
                                                           i64 Kp) {
  __shared__ uint32_t tile[8][PB_TN][PB_ROW];
  __shared__ i64 tap_off[PB_TK];
  __shared__ int tap_r[PB_TK], tap_s[PB_TK], tap_src[PB_TK];  // src: 0 pair 1, 1 pair 2, -1 none
  const mpc_conv_desc& d = cg.d;
  const i64 k0 = (i64)blockIdx.x * PB_TK, n0 = (i64)blockIdx.y * PB_TN;
  const int tid = threadIdx.x, nl = tid & 31, kq = tid >> 5;
  const u64* src2 = cg.src2[job];
  if (tid < PB_TK) {
    i64 k = k0 + tid;
    int src = 0;
    if (k >= K) {
      k -= K;
      src = 1;
    }
    if (k >= K || (src == 1 && !src2)) {
      tap_src[tid] = -1;
      tap_off[tid] = 0;
      tap_r[tid] = tap_s[tid] = 0;
    } else {
      const i64 s_ = k % d.kw, r = (k / d.kw) % d.kh, ci = k / (d.kw * d.kh);
      tap_src[tid] = src;
      tap_off[tid] = (ci * d.h + r) * d.w + s_;
      tap_r[tid] = (int)r;
      tap_s[tid] = (int)s_;
    }
  }
  // Output column n -> (b, oh, ow), and the data offset of its window origin.
  const i64 n = n0 + nl;
  const bool n_ok = n < N;
  const i64 ow = n % cg.wo, oh = (n / cg.wo) % cg.ho, b = n / (cg.wo * cg.ho);
  const i64 oy = oh * d.stride_h - d.pad_h, ox = ow * d.stride_w - d.pad_w;
  const i64 base = (b * d.c_in * d.h + oy) * d.w + ox;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int kl = 2 * (kq + 8 * j);
    u64 v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int t = kl + e;
      const int src = tap_src[t];
      v[e] = 0;
      const i64 y = oy + tap_r[t], x = ox + tap_s[t];
      if (n_ok && src >= 0 && y >= 0 && y < d.h && x >= 0 && x < d.w) {
        const i64 off = base + tap_off[t];
        if (src == 0) {
          u64 acc = 0;
          for (int q = 0; q < cg.n1; ++q) {
            acc += cg.src1[q * cg.stride1 + off];
            if (cg.sub1) acc -= cg.sub1[q * cg.stride1 + off];
          }
          v[e] = acc;
        } else {
          v[e] = src2[off];
        }
      }
    }
    int d0[8], d1[8];
    balanced_digits(v[0], d0);
    balanced_digits(v[1], d1);
#pragma unroll
    for (int pl = 0; pl < 8; ++pl) tile[pl][nl][kl >> 1] = pack_bf16x2(d0[pl], d1[pl]);
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < 8 * PB_TN; r += 8) {
    const int pl = r / PB_TN, row = r % PB_TN;
    const i64 nn = n0 + row;
    const i64 kk = k0 + 2 * lane;
    if (nn < N && kk < Kp)
      *reinterpret_cast<uint32_t*>(out + ((i64)pl * N + nn) * Kp + kk) = tile[pl][row][lane];
  }
}

// ---- host side -----------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode ? MPC_OK : fail(MPC_ECUDA, "cuTensorMapEncodeTiled unavailable");
}

// 3-D map over planes [8][rows][Kp] bf16 with a {16, box_rows, 8} box, 32-byte swizzle.
int encode_planes(CUtensorMap* tm, const void* base, i64 rows, i64 Kp, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 8};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)KS, (cuuint32_t)box_rows, 8};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? MPC_OK : fail(MPC_ECUDA, "tensor map encode failed (%d)", (int)r);
}

inline i64 padded_k(i64 K, int npairs) { return ceil_div(npairs * K, KS) * KS; }

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int limb_splits(i64 M, i64 N, i64 K, int npairs, int njobs) {
  const i64 tiles = ceil_div(M, BM) * ceil_div(N, BN) * njobs;
  return choose_splits(tiles, padded_k(K, npairs) / KS, 32);
}

bool limb_supported(i64 M, i64 N, i64 K) {
  // TMA coordinates are 32-bit; keep every extent comfortably inside.
  return M >= 1 && N >= 1 && K >= 1 && M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 30);
}

size_t limb_workspace_bytes(i64 M, i64 N, i64 K, int npairs, int njobs) {
  const i64 Kp = padded_k(K, npairs);
  return (size_t)njobs * (al256((size_t)8 * M * Kp * 2) + al256((size_t)8 * N * Kp * 2));
}

int launch_gemm_limb(const GemmArgs& g_in, void* ws, size_t ws_bytes, cudaStream_t s) {
  GemmArgs g = g_in;
  if (g.splits < 1) g.splits = 1;
  if (g.M <= 0 || g.N <= 0 || g.njobs <= 0) return MPC_OK;
  if ((g.splits > 1 && g.partial == nullptr) || g.splits * g.njobs > 65535)
    return fail(MPC_EINVAL, "bad split configuration");
  if (!limb_supported(g.M, g.N, g.K)) return fail(MPC_EUNSUPPORTED, "shape outside limb engine");
  if (int rc = get_encoder()) return rc;
  const int npairs = g.jobs[0].A2 ? 2 : 1;
  for (int j = 1; j < g.njobs; ++j)
    if ((g.jobs[j].A2 != nullptr) != (npairs == 2))
      return fail(MPC_EINVAL, "limb engine: jobs mix one- and two-pair products");
  const i64 Kp = padded_k(g.K, npairs);
  const size_t need = limb_workspace_bytes(g.M, g.N, g.K, npairs, g.njobs);
  if (ws == nullptr || ws_bytes < need)
    return fail(MPC_ENOMEM, "limb workspace %zu bytes, need %zu", ws_bytes, need);
  const i64 gy = ceil_div(g.M, BM), gx = ceil_div(g.N, BN);
  if (gy > 65535) return fail(MPC_EUNSUPPORTED, "M too large for the limb engine grid");
  int* st = device_status_ptr();
  if (!st) return fail(MPC_ECUDA, "device status word unavailable");

  // Planes for every job.
  PlaneJob ja[8] = {}, jbv[8] = {};
  char* w = static_cast<char*>(ws);
  LimbParams prm;
  memset(&prm, 0, sizeof(prm));
  for (int j = 0; j < g.njobs; ++j) {
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(w);
    w += al256((size_t)8 * g.M * Kp * 2);
    __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(w);
    w += al256((size_t)8 * g.N * Kp * 2);
    ja[j] = PlaneJob{g.jobs[j].A1, g.jobs[j].A2, pa};
    jbv[j] = PlaneJob{g.jobs[j].B1, g.jobs[j].B2, pb};
    if (int rc = encode_planes(&prm.tmA[j], pa, g.M, Kp, BM)) return rc;
    if (int rc = encode_planes(&prm.tmB[j], pb, g.N, Kp, BN)) return rc;
    prm.C[j] = g.jobs[j].C;
    prm.Z[j] = g.jobs[j].Z;
  }
  {
    KernelTimer timer("limb_planes", s);
    const i64 ta = g.M * (Kp / 8);
    dim3 ga(grid_for(ta, 256, 148 * 16), g.njobs);
    dim3 gb((unsigned)ceil_div(Kp, PB_TK), (unsigned)ceil_div(g.N, PB_TN), g.njobs);
    if (ceil_div(g.N, PB_TN) > 65535) return fail(MPC_EUNSUPPORTED, "N too large for the plane pass");
    limb_planes_a<<<ga, 256, 0, s>>>(ja[0], ja[1], ja[2], ja[3], ja[4], ja[5], ja[6],
                                     ja[7], g.M, g.K, Kp);
    if (int rc = check_launch("limb_planes_a")) return rc;
    if (g.gather) {
      for (int j = 0; j < g.njobs; ++j) {
        dim3 gj(gb.x, gb.y, 1);
        limb_planes_b_conv<<<gj, 256, 0, s>>>(*g.gather, j, jbv[j].out, g.N, g.K, Kp);
        if (int rc = check_launch("limb_planes_b_conv")) return rc;
      }
    } else {
      limb_planes_b<<<gb, 256, 0, s>>>(jbv[0], jbv[1], jbv[2], jbv[3], jbv[4], jbv[5],
                                       jbv[6], jbv[7], g.N, g.K, Kp);
      if (int rc = check_launch("limb_planes_b")) return rc;
    }
  }
  prm.M = g.M;
  prm.N = g.N;
  prm.hw_out = g.hw_out;
  prm.T = (int)(Kp / KS);
  prm.trunc_bits = g.trunc_bits;
  prm.splits = g.splits;
  prm.njobs = g.njobs;
  prm.partial = g.partial;
  prm.status = st;
  cudaError_t e = cudaFuncSetAttribute(limb_gemm_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return fail(MPC_ECUDA, "smem attribute: %s", cudaGetErrorString(e));
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(g.njobs * g.splits));
  {
    KernelTimer timer("gemm_limb", s);
    limb_gemm_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(prm);
    if (int rc = check_launch("gemm_limb")) return rc;
  }
  return g.splits > 1 ? gemm_reduce(g, s) : MPC_OK;
}

}  // namespace mpc
