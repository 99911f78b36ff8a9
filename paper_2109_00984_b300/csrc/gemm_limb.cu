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
//  * pairs with the same shift s = i + j share one fp32 TMEM accumulator.  A
//    tile is 128 x 128 and runs in two passes over its K range: pass 0 the
//    shifts 0..3 (digit planes 0..3 only), pass 1 the shifts 4..7 (all planes),
//    four accumulators of 128 x 128 per pass filling the 512 TMEM columns.
//    With N = 128 an MMA reads 8 KiB of operands from shared memory per
//    128 x 128 x 16 MACs, which the tensor core's shared-memory port sustains at
//    full rate (N = 64 with eight accumulators would read 6 KiB per half the
//    work and cap the tensor pipe near two thirds of its peak);
//  * |d_i d_j| <= 2^14 and shift s sums s + 1 pairs, so 64 / (s + 1)
//    sub-steps of K = 16 (1024 K-steps for shift 0, 128 for shift 7) keep
//    every partial sum within 2^24 where fp32 holds integers exactly.  Each
//    accumulator is drained at the end of such a chunk (chunks staggered by
//    slot) into a 64-bit integer register sum R += int(acc_s) << 8s: 0.58
//    drains per sub-step over both passes, where a common chunk of 8 for
//    every shift would take one;
//  * the epilogue parks the sums in shared memory (the operand stages are idle
//    by then) and writes whole rows: it adds C, applies the optional
//    truncation and stores, or stores the split-K partial.
//
// Operands arrive as digit planes written by limb_planes: A by rows of
// M, B transposed by rows of N (both K-major), interleaved per sub-step: row r
// holds, for each sub-step t of 16 k, the 16 digits of planes 0..7 in turn
// (256 contiguous bytes), i.e. [rows][T][8][16] bf16.  A TMA box is 128 rows x
// 128 bytes (planes 0..3 or 4..7 of one sub-step) with the 128-byte swizzle,
// so the copy engine fetches whole 128-byte lines (a [8][rows][K] layout with
// 32-byte boxes made four times as many L2 requests); the MMA of plane p
// starts 32 (p % 4) bytes into the swizzled rows, as a K-step inside a
// 128-byte swizzle atom would.
// K-concatenated operand pairs (Z = C + A1 B1 + A2 B2) are one GEMM over
// [A1 | A2] and [B1 ; B2], each pair with its own planes.
//
// Warp roles of the one-launch kernel (768 threads): warps 0-3 each issue the
// MMAs of one accumulator slot q (shift q in pass 0, 4 + q in pass 1), one
// thread per warp; one thread of warp 4 issues every TMA load, as soon as a
// stage is released (an MMA issue holds its thread until the tensor pipe takes
// it, so a loader that also issued MMAs delivered its stages late); warps 5-7
// complete that warpgroup; warp 0 allocates TMEM; warps 8-23 drain TMEM, four
// per lane quadrant (warp w reads lanes 32 (w % 4) .. +31), 32 columns each,
// and write the output.  A pass-0 stage holds two sub-steps (planes 0..3 of t
// and of t + 1), so each barrier round trip of pass 0 feeds 20 MMAs.  After
// launch (80 registers per thread) the MMA warpgroup drops to 40, the producer
// warpgroup to 24 and the drain warpgroups rise to 104 (setmaxnreg), so a
// drain can hold a slot's 32 loaded columns beside its 32 64-bit sums and
// release the slot before converting.  Every wait is bounded: on a timeout the
// CTA records MPC_ETIMEOUT, waits (bounded) for its own copies and MMAs, frees
// TMEM and returns.
//
// A persistent variant (limb_gemm_grouped_kernel) runs the tiles of a whole
// batch of Beaver matmuls: one CTA per SM claims 128 x 128 tiles of any
// product and party from an atomic counter, longest K first, with the
// pipeline's barrier phases carried from tile to tile; its digit planes come
// from one grouped plane pass (limb_planes_grouped).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int BM = 128, BN = 128, KS = 16, STAGES = 3, NPLANE = 8, NSLOT = 4;
constexpr int PLANE_BYTES = BM * KS * 2;               // 4 KiB: one digit plane of a tile
constexpr int A_STAGE_BYTES = NPLANE * PLANE_BYTES;    // 32 KiB
constexpr int STAGE_BYTES = 2 * A_STAGE_BYTES;         // A then B planes: 64 KiB
constexpr int HALF_LOAD_BYTES = 4 * PLANE_BYTES;       // one TMA box: 128 rows x 128 B
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
// Warp roles (both kernels, 24 warps): warps 0-3 issue the MMAs of
// accumulator slots 0-3, warp 4 issues the TMA loads, warps 5-7 only complete
// that warpgroup, warps 8-23 drain.  A tcgen05.mma holds its thread until the
// tensor pipe takes it (about 120 cycles for one thread alone, 200+ with four
// competing), so a loader that also issued MMAs delivered each stage late; on
// its own warp it refills a stage as soon as the MMAs release it.
constexpr int kIssuers = 4;        // MMA-issuing warps 0..3, one accumulator slot each
constexpr int kProducerWarp = 4;   // TMA loads (one thread)
constexpr int kDrainBase = 8;      // first TMEM drain / epilogue warp
constexpr int kDrainWarps = 16;
constexpr int kWarps = kDrainBase + kDrainWarps, kThreads = 32 * kWarps;
static_assert(BM % kDrainWarps == 0, "epilogue rows split evenly over the drain warps");
// Launched with 80 registers per thread (768 threads); after launch
// (setmaxnreg) the MMA warpgroup keeps 40, the producer warpgroup 24 and the
// drain warpgroups take 104, enough to hold a slot's 32 drained columns beside
// the 32 64-bit sums.
constexpr int kLaunchRegs = 80, kIssuerRegs = 40, kProducerRegs = 24, kDrainRegs = 104;
static_assert(kIssuers == 4 && kDrainBase % 4 == 0 && kDrainWarps % 4 == 0, "warpgroup-aligned roles");
static_assert(32 * 4 * kIssuerRegs + 32 * 4 * kProducerRegs + 32 * kDrainWarps * kDrainRegs <=
                  kThreads * kLaunchRegs,
              "register split exceeds the launch allocation");
constexpr uint32_t TMEM_COLS = 512;
static_assert(BM == BN, "A and B plane tiles share one layout");
static_assert(BM * (BN + 1) * 8 <= STAGES * STAGE_BYTES, "epilogue tile fits the stages");
// Instruction descriptor, kind::f16: D f32 (bit 4), A bf16 (bits 7-9 = 1),
// B bf16 (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
// The same with N = 64: a grouped tile with at most 64 columns left in its
// product runs half-width MMAs (the accumulator's other 64 columns are never
// written and never stored).
constexpr uint32_t IDESC_N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                               ((uint32_t)(BM >> 4) << 24);
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

// Each operand pair has its own planes ([rows][K1p / 16][8][16], K1p = K
// rounded up to 16), so a pair that all jobs share (the opened E or F) is cut into digits
// once: tmA[pair][job] / tmB[pair][job] of different jobs may map one buffer.
struct LimbParams {
  CUtensorMap tmA[2][MPC_MAX_PARTIES];
  CUtensorMap tmB[2][MPC_MAX_PARTIES];
  const u64* C[MPC_MAX_PARTIES];
  u64* Z[MPC_MAX_PARTIES];
  u64* partial;  // split-K partial sums [splits][njobs][M][N] (splits > 1)
  i64 M, N, hw_out;
  int T;   // K sub-steps of 16 over both pairs
  int T1;  // sub-steps of one pair
  // One-pair jobs of different K (a batch of dealer products): job j's
  // sub-steps when Tj[j] > 0, else T (= T1).
  int Tj[MPC_MAX_PARTIES];
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
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
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // version
  d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
  return d;
}

// Descriptor offset (16-byte units) of digit plane p inside a stage region:
// planes 0..3 in the first 128 x 128-byte box, 4..7 in the second, plane p
// starting 32 (p % 4) bytes into each swizzled row.
__device__ __forceinline__ uint64_t plane_desc_off(int p) {
  return (uint64_t)(((p >> 2) * HALF_LOAD_BYTES + (p & 3) * 32) >> 4);
}

#define TMEM_LD_X16(taddr, r)                                                                  \
  asm volatile(                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "  \
      "%11, %12, %13, %14, %15}, [%16];"                                                        \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),    \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),             \
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                                                  \
      : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The s + 1 digit-pair MMAs of shift s: D += sum_{i <= s} A_i B_{s - i}.
__device__ __forceinline__ void issue_shift(uint32_t d, uint64_t a0, uint64_t b0, int s,
                                            bool start, uint32_t idesc) {
  tc_mma(d, a0, b0 + plane_desc_off(s), idesc, start ? 0u : 1u);
  for (int i = 1; i <= s; ++i)
    tc_mma(d, a0 + plane_desc_off(i), b0 + plane_desc_off(s - i), idesc, 1u);
}

// Chunk length of shift s in sub-steps of K = 16: the shift sums the s + 1
// digit pairs (i, s - i), each product at most 2^14 in magnitude, so
// L_s = 64 / (s + 1) sub-steps keep every partial sum within
// L_s * 16 * (s + 1) * 2^14 <= 2^24 (64, 32, 21, 16, 12, 10, 9, 8).
__device__ __forceinline__ int chunk_len(int s) { return 64 / (s + 1); }

// Sub-steps left, t included, in the chunk of shift s (slot s % 4) that holds
// sub-step t: a chunk ends when (t + s % 4 * L_s / 4) % L_s = L_s - 1, which
// staggers the four slots' drains by a quarter period.  The last sub-step of
// the K range ends every chunk.
__device__ __forceinline__ int chunk_left(int t, int s) {
  const int L = chunk_len(s);
  return L - (t + (s & 3) * L / 4) % L;
}

// Descriptor offset between consecutive stages (16-byte units).
constexpr uint64_t STAGE_DESC = STAGE_BYTES >> 4;

// Copies in flight must land before the CTA can leave (bounded): the last
// load into each stage, out of the n issued.
__device__ __forceinline__ void drain_copies(int n, uint64_t* full_bar) {
  for (int i = 0; i < STAGES && i < n; ++i) {
    const int last = n - 1 - ((n - 1 - i) % STAGES);
    const uint32_t ph = (uint32_t)(last / STAGES) & 1u;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(&full_bar[i], ph) && globaltimer() - t0 < kWaitLimitNs) {
    }
  }
}

// The producer (warp 4, one thread): every load of the CTA's sub-steps in
// order, each as soon as its stage is released, so STAGES stages are in
// flight.  A pass-0 stage carries two sub-steps (digit planes 0..3 of t where
// a pass-1 stage keeps planes 0..3, those of t + 1 where it keeps 4..7), so
// every barrier round trip of pass 0 feeds 20 MMAs instead of 10.
__device__ __forceinline__ void producer_loop(const LimbParams& p, int job, int m0, int n0,
                                              uint32_t sbase, int t_begin, int t_end,
                                              uint64_t* full_bar, uint64_t* empty_bar,
                                              volatile int* abort_flag) {
  const CUtensorMap* ta[2] = {&p.tmA[0][job], &p.tmA[1][job]};
  const CUtensorMap* tb[2] = {&p.tmB[0][job], &p.tmB[1][job]};
  const int T1 = p.Tj[job] > 0 ? p.Tj[job] : p.T1;
  int st = 0, n = 0;
  uint32_t ph = 0;
  // One box of digit planes (plane group h: 0..3 or 4..7) of sub-step t of A
  // and of B, into the two halves at offset `half` of the stage.
  auto box = [&](int t, int h, uint32_t half) {
    const int pair = t >= T1;
    const int tl = pair ? t - T1 : t;
    const uint32_t a_dst = sbase + (uint32_t)st * STAGE_BYTES + half;
    tma_load_4d(a_dst, pair ? ta[1] : ta[0], &full_bar[st], 0, h, tl, m0);
    tma_load_4d(a_dst + A_STAGE_BYTES, pair ? tb[1] : tb[0], &full_bar[st], 0, h, tl, n0);
  };
  auto next = [&]() {
    ++n;
    if (++st == STAGES) {
      st = 0;
      ph ^= 1u;
    }
  };
  bool ok = true;
  for (int t = t_begin; t < t_end && ok; t += 2) {
    const bool two = t + 1 < t_end;
    if (!(ok = mbar_wait(&empty_bar[st], ph ^ 1u, abort_flag))) break;
    mbar_arrive_expect_tx(&full_bar[st], (two ? 4 : 2) * HALF_LOAD_BYTES);
    box(t, 0, 0);
    if (two) box(t + 1, 0, HALF_LOAD_BYTES);
    next();
  }
  for (int t = t_begin; t < t_end && ok; ++t) {
    if (!(ok = mbar_wait(&empty_bar[st], ph ^ 1u, abort_flag))) break;
    mbar_arrive_expect_tx(&full_bar[st], 4 * HALF_LOAD_BYTES);
    box(t, 0, 0);
    box(t, 1, HALF_LOAD_BYTES);
    next();
  }
  drain_copies(n, full_bar);
}

// One accumulator slot's MMA schedule: shift q in pass 0, 4 + q in pass 1; a
// chunk starts at the range's first sub-step or right after the previous one
// ended, and first waits until the drain warps have read the slot's previous
// chunk (which may belong to pass 0).
struct Slot {
  uint32_t d;       // TMEM address of the accumulator
  int q, shift, len, left;
  bool start;
  uint32_t chunks;  // chunks committed so far
  uint32_t idesc;   // instruction descriptor: N = 128, or 64 for a narrow grouped tile
  __device__ __forceinline__ void begin_pass(int pass, int t_begin, uint32_t tmem) {
    d = tmem + (uint32_t)(q * BN);
    shift = 4 * pass + q;
    len = chunk_len(shift);
    left = chunk_left(t_begin, shift);
    start = true;
  }
  // The slot's MMAs of one sub-step; false on an abort.
  __device__ __forceinline__ bool step(uint64_t a0, uint64_t b0, bool last, uint64_t* accf_bar,
                                       uint64_t* acce_bar, volatile int* abort_flag) {
    if (start && chunks > 0) {
      if (!mbar_wait(&acce_bar[q], (chunks - 1u) & 1u, abort_flag)) return false;
      tc_fence_after();
    }
    issue_shift(d, a0, b0, shift, start, idesc);
    start = --left == 0 || last;
    if (start) {
      tc_commit(&accf_bar[q]);
      chunks++;
      left = len;
    }
    return true;
  }
};

// MMA issuer of accumulator slot q (warp q): pass 0 two sub-steps per stage
// (the second one's planes 0..3 where pass 1 keeps planes 4..7), pass 1 one;
// the stage and its phase are kept as counters.
__device__ __forceinline__ void mma_loop(int q, uint32_t sbase, uint32_t tmem, int t_begin,
                                         int t_end, uint64_t* full_bar, uint64_t* empty_bar,
                                         uint64_t* accf_bar, uint64_t* acce_bar,
                                         volatile int* abort_flag) {
  Slot sl{0, q, 0, 0, 0, true, 0u, IDESC};
  const uint64_t a_base = smem_desc_sw128(sbase);
  const uint64_t b_base = smem_desc_sw128(sbase + A_STAGE_BYTES);
  constexpr uint64_t HALF_DESC = HALF_LOAD_BYTES >> 4;
  int st = 0;
  uint32_t ph = 0;
  auto next = [&]() {
    if (++st == STAGES) {
      st = 0;
      ph ^= 1u;
    }
  };
  sl.begin_pass(0, t_begin, tmem);
  for (int t = t_begin; t < t_end; t += 2) {
    if (!mbar_wait(&full_bar[st], ph, abort_flag)) return;
    tc_fence_after();
    const uint64_t a0 = a_base + (uint64_t)st * STAGE_DESC;
    const uint64_t b0 = b_base + (uint64_t)st * STAGE_DESC;
    if (!sl.step(a0, b0, t == t_end - 1, accf_bar, acce_bar, abort_flag)) return;
    if (t + 1 < t_end &&
        !sl.step(a0 + HALF_DESC, b0 + HALF_DESC, t + 1 == t_end - 1, accf_bar, acce_bar, abort_flag))
      return;
    tc_commit(&empty_bar[st]);
    next();
  }
  sl.begin_pass(1, t_begin, tmem);
  for (int t = t_begin; t < t_end; ++t) {
    if (!mbar_wait(&full_bar[st], ph, abort_flag)) return;
    tc_fence_after();
    const uint64_t a0 = a_base + (uint64_t)st * STAGE_DESC;
    const uint64_t b0 = b_base + (uint64_t)st * STAGE_DESC;
    if (!sl.step(a0, b0, t == t_end - 1, accf_bar, acce_bar, abort_flag)) return;
    tc_commit(&empty_bar[st]);
    next();
  }
}

__global__ void __launch_bounds__(kThreads, 1) limb_gemm_kernel(const __grid_constant__ LimbParams p) {
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[NSLOT], acce_bar[NSLOT], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int job = blockIdx.z / p.splits, split = blockIdx.z % p.splits;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // This CTA's K sub-steps [t_begin, t_end), run once per pass.
  const int T = p.Tj[job] > 0 ? p.Tj[job] : p.T;
  const int t_begin = (int)((i64)T * split / p.splits);
  const int t_end = (int)((i64)T * (split + 1) / p.splits);
  const uint32_t sbase = (smem_u32(dsmem) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], kIssuers);
    }
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&accf_bar[i], 1);
      mbar_init(&acce_bar[i], kDrainWarps);
    }
    mbar_init(&done_bar, kIssuers);
    // A timeout recorded by an earlier CTA (and not yet cleared by
    // mpc_sync_status) makes every later CTA skip its work and exit at once.
    abort_flag = (*(volatile int*)p.status == MPC_ETIMEOUT) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int pr = 0; pr < 2; ++pr) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.tmA[pr][job])));
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.tmB[pr][job])));
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < kIssuers) {
    // The MMA and producer warpgroups hand registers to the drain warpgroups:
    // 128 x 40 + 128 x 24 + 512 x 104 = 61 440 = 768 x 80 launched.
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kIssuerRegs));
    if (lane == 0) {
      // ---- MMA issuers: warp q owns accumulator slot q ----
      mma_loop(warp, sbase, tmem, t_begin, t_end, full_bar, empty_bar, accf_bar, acce_bar,
               &abort_flag);
      // All of this issuer's MMAs must finish before TMEM is released (bounded).
      tc_commit(&done_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&done_bar, 0) && globaltimer() - t0 < kWaitLimitNs) {
      }
    }
  } else if (warp < kDrainBase) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
    // ---- the producer: TMA loads only ----
    if (warp == kProducerWarp && lane == 0)
      producer_loop(p, job, m0, n0, sbase, t_begin, t_end, full_bar, empty_bar, &abort_flag);
  } else {
    // ---- TMEM drain + epilogue: 16 warps, four per TMEM lane quadrant ----
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kDrainRegs));
    const int ew = warp - kDrainBase;          // 0..15
    const int quad = warp & 3;                    // lane quadrant this warp may access
    const int cblk = ew >> 2;                     // which 32 of the 128 columns
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cblk * 32);
    u64 R[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) R[j] = 0;
    uint32_t parity = 0;  // bit q: parity of the next chunk of slot q
    bool ok = true;
    // Drain slot q's finished chunk of shift sh / 8 into R.
    // R[j] += int(acc) << sh for 16 columns.  From shift 4 on (sh >= 32) only
    // the upper word changes: one 32-bit shift-add per value.
    auto accumulate = [&](const uint32_t (&v)[16], u64* Rh, int sh) {
      if (sh >= 32) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t iv = (uint32_t)__float2int_rz(__uint_as_float(v[j]));
          const uint32_t hi = (uint32_t)(Rh[j] >> 32) + (iv << (sh - 32));
          Rh[j] = (Rh[j] & 0xFFFFFFFFull) | ((u64)hi << 32);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int iv = __float2int_rz(__uint_as_float(v[j]));
          Rh[j] += (u64)(i64)iv << sh;
        }
      }
    };
    // Drain slot q's finished chunk of shift sh / 8 into R.  The slot is
    // released to its issuer as soon as both 16-column loads have landed, so
    // the conversions overlap the next chunk's MMAs (the 32 loaded columns
    // beside R need the drain warps' larger register share).
    auto drain = [&](int q, int sh) -> bool {
      if (!mbar_wait(&accf_bar[q], (parity >> q) & 1u, &abort_flag)) return false;
      tc_fence_after();
      uint32_t v[16], w[16];
      TMEM_LD_X16(lane_base + (uint32_t)(q * BN), v);
      TMEM_LD_X16(lane_base + (uint32_t)(q * BN + 16), w);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[q]);
      accumulate(v, R, sh);
      accumulate(w, R + 16, sh);
      parity ^= 1u << q;
      return true;
    };
    for (int pass = 0; pass < 2 && ok; ++pass) {
      // Byte q: sub-steps left in slot q's chunk (1..64), all four decremented
      // together; a byte that reaches 0 is refilled with the chunk length.
      uint32_t left = 0;
#pragma unroll
      for (int q = 0; q < NSLOT; ++q) left |= (uint32_t)chunk_left(t_begin, 4 * pass + q) << (8 * q);
      for (int t = t_begin; t < t_end && ok; ++t) {
        left -= 0x01010101u;
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) {
          if (((left >> (8 * q)) & 0xFFu) == 0u || t == t_end - 1) {
            if (ok) ok = drain(q, 8 * (4 * pass + q));
            left |= (uint32_t)chunk_len(4 * pass + q) << (8 * q);
          }
        }
      }
    }
    // Epilogue through shared memory (the operand stages are idle once every
    // chunk is drained): each thread parks its 32 sums of one row, then each
    // warp writes whole rows, 256 contiguous bytes per store instruction,
    // instead of 32 rows x 8 bytes.  Rows of 129 words keep the parking
    // stores at the two wavefronts that 256 bytes need.
    constexpr int SROW = BN + 1;
    u64* stile = reinterpret_cast<u64*>(dsmem + (sbase - smem_u32(dsmem)));
    if (ok && !abort_flag) {
      u64* mine = stile + (quad * 32 + lane) * SROW + cblk * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) mine[j] = R[j];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kDrainWarps) : "memory");
    if (!abort_flag) {
      for (int r = ew; r < BM; r += kDrainWarps) {
        const i64 row = (i64)m0 + r;
        if (row >= p.M) break;
        const u64* src = stile + r * SROW;
        if (p.splits > 1) {
          u64* part = p.partial + ((i64)split * p.njobs + job) * p.M * p.N + row * p.N;
#pragma unroll
          for (int k = 0; k < BN / 32; ++k) {
            const int c = 32 * k + lane;
            if ((i64)n0 + c < p.N) part[n0 + c] = src[c];
          }
        } else {
          const u64* C = p.C[job];
          u64* Z = p.Z[job];
#pragma unroll
          for (int k = 0; k < BN / 32; ++k) {
            const int c = 32 * k + lane;
            const i64 col = (i64)n0 + c;
            if (col < p.N) {
              const i64 idx = gemm_out_index(row, col, p.M, p.N, p.hw_out);
              u64 v = src[c];
              if (C) v += C[idx];
              if (p.trunc_bits > 0) v = sar(v, p.trunc_bits);
              Z[idx] = v;
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) record_status(p.status, MPC_ETIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}


// ---- persistent grouped engine ------------------------------------------------------------
// The same tile algorithm as limb_gemm_kernel, restated as per-tile functions
// whose pipeline state carries over from one tile to the next, so that one
// CTA per SM can run tile after tile of many products (a batch of Beaver
// matmuls) in one launch.  The one-launch kernel above keeps its own copy:
// measured against these functions it is about 5 % faster on single GEMMs.
//
// What one CTA computes for one output tile: the operand planes' tensor maps
// per pair, its K sub-steps [t_begin, t_end) over both pairs (run once per
// pass), and where the sums go.
struct TileJob {
  const CUtensorMap* ta[2];  // A planes of pair 0 and pair 1
  const CUtensorMap* tb[2];  // B planes of pair 0 and pair 1
  const u64* C;              // added in the epilogue (null: none)
  u64* Z;                    // output
  u64* part;                 // split-K: raw partial tile destination [M][N] instead of Z
  i64 M, N, hw_out;
  int m0, n0;
  int T1;                    // sub-steps of one pair
  int t_begin, t_end;
  int trunc_bits;
};

// Barriers and buffers of a persistent CTA (at namespace scope, so their
// shared-memory addresses are constants).  Barrier phases run on across its
// tiles: sub-steps are numbered from the CTA's
// first tile on (the stage of global sub-step G is G % STAGES, its phase
// (G / STAGES) & 1), the issuers count their chunks and the drain warps keep
// one phase bit per slot.
extern __shared__ __align__(1024) uint8_t gq_smem[];
__shared__ __align__(8) uint64_t gq_full[STAGES], gq_empty[STAGES];
__shared__ __align__(8) uint64_t gq_accf[NSLOT], gq_acce[NSLOT], gq_done;
__shared__ uint32_t gq_tmem_slot;
__shared__ volatile int gq_abort;
// The current and the next tile's job (double-buffered: the next one is
// claimed and decoded while the current one runs); in registers beside the
// drain sums they would spill.
__shared__ TileJob gq_job[2];
__shared__ long long gq_item[2];

// Stage buffers: 1024-byte aligned start of the dynamic shared memory.
__device__ __forceinline__ uint32_t stage_base() { return (smem_u32(gq_smem) + 1023u) & ~1023u; }

// The loads of one tile of the grouped launch (the producer thread), in the
// order of the one-launch kernel: pass-0 stages of two sub-steps, pass-1
// stages of one.  The stage, its phase and the count of stage uses run on
// from tile to tile.  False on an abort.
__device__ __forceinline__ bool producer_tile(const TileJob& jb, int& st, uint32_t& ph, int& n) {
  const CUtensorMap* ta[2] = {jb.ta[0], jb.ta[1]};
  const CUtensorMap* tb[2] = {jb.tb[0], jb.tb[1]};
  const int m0 = jb.m0, n0 = jb.n0, T1 = jb.T1, t_begin = jb.t_begin, t_end = jb.t_end;
  const uint32_t sbase = stage_base();
  auto box = [&](int t, int h, uint32_t half) {
    const int pair = t >= T1;
    const int tl = pair ? t - T1 : t;
    const uint32_t a_dst = sbase + (uint32_t)st * STAGE_BYTES + half;
    tma_load_4d(a_dst, pair ? ta[1] : ta[0], &gq_full[st], 0, h, tl, m0);
    tma_load_4d(a_dst + A_STAGE_BYTES, pair ? tb[1] : tb[0], &gq_full[st], 0, h, tl, n0);
  };
  auto next = [&]() {
    ++n;
    if (++st == STAGES) {
      st = 0;
      ph ^= 1u;
    }
  };
  for (int t = t_begin; t < t_end; t += 2) {
    const bool two = t + 1 < t_end;
    if (!mbar_wait(&gq_empty[st], ph ^ 1u, &gq_abort)) return false;
    mbar_arrive_expect_tx(&gq_full[st], (two ? 4 : 2) * HALF_LOAD_BYTES);
    box(t, 0, 0);
    if (two) box(t + 1, 0, HALF_LOAD_BYTES);
    next();
  }
  for (int t = t_begin; t < t_end; ++t) {
    if (!mbar_wait(&gq_empty[st], ph ^ 1u, &gq_abort)) return false;
    mbar_arrive_expect_tx(&gq_full[st], 4 * HALF_LOAD_BYTES);
    box(t, 0, 0);
    box(t, 1, HALF_LOAD_BYTES);
    next();
  }
  return true;
}

// The MMAs of one tile for accumulator slot sl.q (one thread of warp q), in
// the producer's stage order; the slot's chunk count (for the drain barrier's
// parity), the stage and its phase run on from tile to tile.  False on an
// abort.
__device__ __forceinline__ bool mma_tile(Slot& sl, uint32_t tmem, const TileJob& jb, int& st,
                                         uint32_t& ph) {
  sl.idesc = jb.N - jb.n0 <= 64 ? IDESC_N64 : IDESC;
  const int t_begin = jb.t_begin, t_end = jb.t_end;
  const uint32_t sbase = stage_base();
  const uint64_t a_base = smem_desc_sw128(sbase);
  const uint64_t b_base = smem_desc_sw128(sbase + A_STAGE_BYTES);
  constexpr uint64_t HALF_DESC = HALF_LOAD_BYTES >> 4;
  auto next = [&]() {
    if (++st == STAGES) {
      st = 0;
      ph ^= 1u;
    }
  };
  sl.begin_pass(0, t_begin, tmem);
  for (int t = t_begin; t < t_end; t += 2) {
    if (!mbar_wait(&gq_full[st], ph, &gq_abort)) return false;
    tc_fence_after();
    const uint64_t a0 = a_base + (uint64_t)st * STAGE_DESC;
    const uint64_t b0 = b_base + (uint64_t)st * STAGE_DESC;
    if (!sl.step(a0, b0, t == t_end - 1, gq_accf, gq_acce, &gq_abort)) return false;
    if (t + 1 < t_end &&
        !sl.step(a0 + HALF_DESC, b0 + HALF_DESC, t + 1 == t_end - 1, gq_accf, gq_acce, &gq_abort))
      return false;
    tc_commit(&gq_empty[st]);
    next();
  }
  sl.begin_pass(1, t_begin, tmem);
  for (int t = t_begin; t < t_end; ++t) {
    if (!mbar_wait(&gq_full[st], ph, &gq_abort)) return false;
    tc_fence_after();
    const uint64_t a0 = a_base + (uint64_t)st * STAGE_DESC;
    const uint64_t b0 = b_base + (uint64_t)st * STAGE_DESC;
    if (!sl.step(a0, b0, t == t_end - 1, gq_accf, gq_acce, &gq_abort)) return false;
    tc_commit(&gq_empty[st]);
    next();
  }
  return true;
}

// TMEM drain and epilogue of one tile by the 16 drain warps (ew = 0..15, four
// per TMEM lane quadrant).  parity: bit q = phase of slot q's next chunk, kept
// across tiles.  Returns false on an abort (nothing is written then).
__device__ __forceinline__ bool drain_tile(uint32_t tmem, const TileJob& jb, uint32_t& parity,
                                           int warp, int lane) {
  const int ew = warp - kDrainBase;             // 0..15
  const int quad = warp & 3;                    // lane quadrant this warp may access
  const int cblk = ew >> 2;                     // which 32 of the 128 columns
  const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cblk * 32);
  u64 R[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) R[j] = 0;
  bool ok = true;
  // R[j] += int(acc) << sh for 16 columns.  From shift 4 on (sh >= 32) only
  // the upper word changes: one 32-bit shift-add per value.
  auto accumulate = [&](const uint32_t (&v)[16], u64* Rh, int sh) {
    if (sh >= 32) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t iv = (uint32_t)__float2int_rz(__uint_as_float(v[j]));
        const uint32_t hi = (uint32_t)(Rh[j] >> 32) + (iv << (sh - 32));
        Rh[j] = (Rh[j] & 0xFFFFFFFFull) | ((u64)hi << 32);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int iv = __float2int_rz(__uint_as_float(v[j]));
        Rh[j] += (u64)(i64)iv << sh;
      }
    }
  };
  // Drain slot q's finished chunk of shift sh / 8 into R.  The slot is
  // released to its issuer as soon as both 16-column loads have landed, so
  // the conversions overlap the next chunk's MMAs (the 32 loaded columns
  // beside R need the drain warps' larger register share).
  auto drain = [&](int q, int sh) -> bool {
    if (!mbar_wait(&gq_accf[q], (parity >> q) & 1u, &gq_abort)) return false;
    tc_fence_after();
    uint32_t v[16], w[16];
    TMEM_LD_X16(lane_base + (uint32_t)(q * BN), v);
    TMEM_LD_X16(lane_base + (uint32_t)(q * BN + 16), w);
    tmem_wait_ld();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&gq_acce[q]);
    accumulate(v, R, sh);
    accumulate(w, R + 16, sh);
    parity ^= 1u << q;
    return true;
  };
  const int t_begin = jb.t_begin, t_end = jb.t_end;
  for (int pass = 0; pass < 2 && ok; ++pass) {
    // Byte q: sub-steps left in slot q's chunk (1..64), all four decremented
    // together; a byte that reaches 0 is refilled with the chunk length.
    uint32_t left = 0;
#pragma unroll
    for (int q = 0; q < NSLOT; ++q) left |= (uint32_t)chunk_left(t_begin, 4 * pass + q) << (8 * q);
    for (int t = t_begin; t < t_end && ok; ++t) {
      left -= 0x01010101u;
#pragma unroll
      for (int q = 0; q < NSLOT; ++q) {
        if (((left >> (8 * q)) & 0xFFu) == 0u || t == t_end - 1) {
          if (ok) ok = drain(q, 8 * (4 * pass + q));
          left |= (uint32_t)chunk_len(4 * pass + q) << (8 * q);
        }
      }
    }
  }
  // Epilogue through shared memory (the operand stages are idle once every
  // chunk is drained): each thread parks its 32 sums of one row, then each
  // warp writes whole rows, 256 contiguous bytes per store instruction,
  // instead of 32 rows x 8 bytes.  Rows of 129 words keep the parking
  // stores at the two wavefronts that 256 bytes need.
  constexpr int SROW = BN + 1;
  u64* stile = reinterpret_cast<u64*>(gq_smem + (stage_base() - smem_u32(gq_smem)));
  if (ok && !gq_abort) {
    u64* mine = stile + (quad * 32 + lane) * SROW + cblk * 32;
#pragma unroll
    for (int j = 0; j < 32; ++j) mine[j] = R[j];
  }
  asm volatile("bar.sync 1, %0;" ::"r"(32 * kDrainWarps) : "memory");
  // The stage buffers are written again by the next tile's TMA loads (async
  // proxy) after the CTA's tile barrier: order this thread's generic accesses
  // to them first.
  if (gq_abort) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    return false;
  }
  // The job's fields in registers: stores through the generic output
  // pointers could alias the shared-memory job and would force reloads.
  const i64 M = jb.M, N = jb.N, hw_out = jb.hw_out;
  const int m0 = jb.m0, n0 = jb.n0, trunc_bits = jb.trunc_bits;
  const u64* __restrict__ C = jb.C;
  u64* __restrict__ Z = jb.Z;
  u64* part0 = jb.part;
  constexpr int ROWS = BM / kDrainWarps, COLS = BN / 32;  // 8 rows of 4 x 32 columns per warp
  if (part0) {
    for (int r = ew; r < BM; r += kDrainWarps) {
      const i64 row = (i64)m0 + r;
      if (row >= M) break;
      const u64* src = stile + r * SROW;
      u64* part = part0 + row * N;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const int c = 32 * k + lane;
        if ((i64)n0 + c < N) part[n0 + c] = src[c];
      }
    }
  } else {
    // Every C word of the warp's rows is requested before the first store, so
    // their latencies overlap (row by row, each store waited for its load).
    u64 cv[ROWS][COLS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      const i64 row = (i64)m0 + ew + i * kDrainWarps;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const i64 col = (i64)n0 + 32 * k + lane;
        cv[i][k] = (C && row < M && col < N) ? C[gemm_out_index(row, col, M, N, hw_out)] : 0ull;
      }
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      const int r = ew + i * kDrainWarps;
      const i64 row = (i64)m0 + r;
      const u64* src = stile + r * SROW;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const int c = 32 * k + lane;
        const i64 col = (i64)n0 + c;
        if (row < M && col < N) {
          u64 v = src[c] + cv[i][k];
          if (trunc_bits > 0) v = sar(v, trunc_bits);
          Z[gemm_out_index(row, col, M, N, hw_out)] = v;
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  return true;
}

// CTA set-up: barriers (thread 0), the abort flag from the device status
// word, TMEM (warp 0, all 512 columns).
__device__ __forceinline__ void cta_setup(const int* status, int warp) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&gq_full[i], 1);
      mbar_init(&gq_empty[i], kIssuers);
    }
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&gq_accf[i], 1);
      mbar_init(&gq_acce[i], kDrainWarps);
    }
    mbar_init(&gq_done, kIssuers);
    // A timeout recorded by an earlier CTA (and not yet cleared by
    // mpc_sync_status) makes every later CTA skip its work and exit at once.
    gq_abort = (*(const volatile int*)status == MPC_ETIMEOUT) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&gq_tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}

// End of an issuer's work in the CTA: all its MMAs must finish before TMEM is
// released (bounded).
__device__ __forceinline__ void issuer_finish() {
  tc_commit(&gq_done);
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(&gq_done, 0) && globaltimer() - t0 < kWaitLimitNs) {
  }
}

__device__ __forceinline__ void cta_teardown(int* status, uint32_t tmem, int warp) {
  tc_fence_before();
  __syncthreads();
  if (gq_abort && threadIdx.x == 0) record_status(status, MPC_ETIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---- the grouped launch: every tile of many products ---------------------------------------
// One product of a grouped launch, as stored in device memory.  Its tiles are
// P x tiles_m x tiles_n work items (party-major), numbered from tile_base;
// party p's GEMM is Z_p = C_p + A1 B1_p + A2_p B2 over the K-concatenated
// pairs, with the digit planes' tensor maps at maps: A side E (pair 1, all
// parties), A_0 .. A_{P-1} (pair 2); then B side G = B_0 + F (pair 1, party 0),
// B_1 .. B_{P-1} (pair 1), F (pair 2, all parties) -- 2 (P + 1) maps.
struct GroupProd {
  i64 M, N;
  i64 tile_base;
  int tiles_m, tiles_n;
  int T1, P;
  const u64* C;
  u64* Z;
  const CUtensorMap* maps;
};

struct GroupParams {
  const GroupProd* prods;
  int count;
  i64 total;                      // work items over all products
  unsigned long long* counter;    // next work item (zeroed by the caller)
  int trunc_bits;
  int* status;
};

// Work item -> tile job: the last product whose tile_base <= item.
__device__ __forceinline__ void group_job(const GroupParams& gp, i64 item, TileJob& jb) {
  int lo = 0, hi = gp.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gp.prods[mid].tile_base <= item) lo = mid; else hi = mid - 1;
  }
  const GroupProd& b = gp.prods[lo];
  const i64 local = item - b.tile_base;
  const i64 per_party = (i64)b.tiles_m * b.tiles_n;
  const int p = (int)(local / per_party);
  const i64 r = local % per_party;
  jb.ta[0] = b.maps;
  jb.ta[1] = b.maps + 1 + p;
  jb.tb[0] = b.maps + (b.P + 1) + p;
  jb.tb[1] = b.maps + 2 * b.P + 1;
  jb.C = b.C + (i64)p * b.M * b.N;
  jb.Z = b.Z + (i64)p * b.M * b.N;
  jb.part = nullptr;
  jb.M = b.M;
  jb.N = b.N;
  jb.hw_out = 0;
  jb.m0 = (int)(r / b.tiles_n) * BM;
  jb.n0 = (int)(r % b.tiles_n) * BN;
  jb.T1 = b.T1;
  jb.t_begin = 0;
  jb.t_end = 2 * b.T1;
  jb.trunc_bits = gp.trunc_bits;
}

// Persistent: one CTA per SM claims work items from an atomic counter until
// none is left (items are laid out longest K first).  Between two tiles all
// roles meet at a CTA barrier: the drain warps' epilogue must have left the
// stage buffers before the next tile's loads overwrite them.  The tensor maps
// live in global memory (written by an earlier kernel of the call): each is
// acquired for the tensor-map proxy before its first use by this CTA.
__global__ void __launch_bounds__(kThreads, 1) limb_gemm_grouped_kernel(
    const __grid_constant__ GroupParams gp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cta_setup(gp.status, warp);
  // Claims a work item into job buffer `buf` (one thread).
  auto claim = [&](int buf) {
    const long long item = gq_abort ? gp.total : (long long)atomicAdd(gp.counter, 1ull);
    gq_item[buf] = item;
    if (item < gp.total) group_job(gp, item, gq_job[buf]);
  };
  if (threadIdx.x == 0) claim(0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = gq_tmem_slot;

  // Tile k runs job buffer k & 1.  At its start the first drain warp claims
  // tile k + 1 into the other buffer (the drain warps idle until the first
  // chunk ends); the CTA barrier at the end of tile k both frees the stage
  // buffers and publishes tile k + 1.
  if (warp < kIssuers) {
    // ---- MMA issuers: warp q owns accumulator slot q ----
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kIssuerRegs));
    Slot sl{0, warp, 0, 0, 0, true, 0u, IDESC};
    int st = 0;
    uint32_t ph = 0;
    for (int k = 0;; ++k) {
      const int buf = k & 1;
      if (gq_item[buf] >= gp.total) break;
      if (lane == 0 && !gq_abort) mma_tile(sl, tmem, gq_job[buf], st, ph);
      __syncwarp();
      asm volatile("bar.sync 2, %0;" ::"r"(kThreads) : "memory");  // tile done, next published
    }
    if (lane == 0) issuer_finish();
  } else if (warp < kDrainBase) {
    // ---- the producer (one thread of warp 4) ----
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
    int st = 0, n = 0;
    uint32_t ph = 0;
    for (int k = 0;; ++k) {
      const int buf = k & 1;
      if (gq_item[buf] >= gp.total) break;
      if (warp == kProducerWarp && lane == 0 && !gq_abort) {
        const TileJob& jb = gq_job[buf];
        for (int pr = 0; pr < 2; ++pr) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                           reinterpret_cast<uint64_t>(jb.ta[pr]))
                       : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                           reinterpret_cast<uint64_t>(jb.tb[pr]))
                       : "memory");
        }
        producer_tile(jb, st, ph, n);
      }
      __syncwarp();
      asm volatile("bar.sync 2, %0;" ::"r"(kThreads) : "memory");
    }
    if (warp == kProducerWarp && lane == 0) drain_copies(n, gq_full);
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kDrainRegs));
    uint32_t parity = 0;
    for (int k = 0;; ++k) {
      const int buf = k & 1;
      if (gq_item[buf] >= gp.total) break;
      if (warp == kDrainBase && lane == 0) claim(buf ^ 1);
      __syncwarp();
      // Always entered: drain_tile's named barrier needs all 16 drain warps
      // (after an abort its waits give up at once and nothing is written).
      drain_tile(tmem, gq_job[buf], parity, warp, lane);
      asm volatile("bar.sync 2, %0;" ::"r"(kThreads) : "memory");
    }
  }
  cta_teardown(gp.status, tmem, warp);
}

// ---- plane pre-pass ---------------------------------------------------------------------
// Balanced base-256 digits of v: v = sum_i d_i 2^(8i) mod 2^64, d_i in [-128, 127].
// With u = v + 0x8080808080808080 (mod 2^64), byte i of u is d_i + 128: adding
// 128 to every digit position absorbs all the carries of the balanced form.
// For a byte b, the float with bits 0x4B000000 | b is 2^23 + b; subtracting
// 2^23 + 128 gives d = b - 128 exactly, and since |d| <= 128 has at most 8
// significant bits its bf16 is the upper half of that float.  digit_bits(u, i)
// returns those float bits (bf16 in the upper 16 bits).
__device__ __forceinline__ uint32_t digit_bits(u64 u, int i) {
  const uint32_t w = (uint32_t)(u >> (i < 4 ? 0 : 32));
  // bytes, high to low: 0x4B, 0, 0, byte (i mod 4) of w
  const uint32_t f = __byte_perm(w, 0x4B000000u, 0x7440u | (uint32_t)(i & 3));
  return __float_as_uint(__uint_as_float(f) - 8388736.0f);
}

__device__ __forceinline__ u64 digit_base(u64 v) { return v + 0x8080808080808080ull; }

// Two bf16 digits packed low | high from their float bits.
__device__ __forceinline__ uint32_t pack_hi16(uint32_t lo_bits, uint32_t hi_bits) {
  return __byte_perm(lo_bits, hi_bits, 0x7632u);
}

// Element offset of digit (plane p, row, k) in interleaved planes
// [rows][Kp / 16][8][16] (Kp a multiple of 16).
__device__ __forceinline__ i64 plane_index(int p, i64 row, i64 Kp, i64 k) {
  return ((row * (Kp / KS) + k / KS) * NPLANE + p) * KS + (k % KS);
}

// Writes 8 consecutive k' (k0 a multiple of 8) of one row into its 8 digit
// planes: eight 16-byte stores, 32 bytes apart.
__device__ __forceinline__ void write_planes(const u64 v[8], __nv_bfloat16* out, i64 row, i64 Kp,
                                             i64 k0) {
  u64 u[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) u[e] = digit_base(v[e]);
#pragma unroll
  for (int pl = 0; pl < 8; ++pl) {
    uint4 w;
    w.x = pack_hi16(digit_bits(u[0], pl), digit_bits(u[1], pl));
    w.y = pack_hi16(digit_bits(u[2], pl), digit_bits(u[3], pl));
    w.z = pack_hi16(digit_bits(u[4], pl), digit_bits(u[5], pl));
    w.w = pack_hi16(digit_bits(u[6], pl), digit_bits(u[7], pl));
    *reinterpret_cast<uint4*>(out + plane_index(pl, row, Kp, k0)) = w;
  }
}

struct PlaneJob {
  const u64* X1;  // first pair operand
  const u64* X2;  // second pair operand (or null)
  __nv_bfloat16* out;
};

struct PlaneJobs {
  PlaneJob j[2 * MPC_MAX_PARTIES];
};

// Element source of the per-GEMM plane pass: the word at index i.
struct DirectSrc {
  const u64* X;
  __device__ __forceinline__ u64 operator()(i64 i) const { return X[i]; }
};

// A side: the source is [M][K] row-major.  Block `blk` of `nblk` strides over
// the 8-k groups; planes go to `out`.
template <class Src>
__device__ __forceinline__ void planes_a_part(const Src& src, __nv_bfloat16* out, i64 M, i64 K,
                                              i64 Kp, i64 blk, i64 nblk) {
  const i64 kc = Kp / 8;
  const i64 total = M * kc;
  for (i64 i = blk * (i64)blockDim.x + threadIdx.x; i < total; i += nblk * blockDim.x) {
    const i64 m = i / kc, k0 = (i % kc) * 8;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const i64 k = k0 + e;
      v[e] = k < K ? src(m * K + k) : 0ull;
    }
    write_planes(v, out, m, Kp, k0);
  }
}

// B side from a row-major [K][N] source, K-major like the convolution gather
// below: lane l of warp w owns column n = 16 by + l / 2 and the 8 consecutive
// k of half l % 2 of sub-step t = 8 bx + w, reads them (16 consecutive n per
// warp and k: whole 128-byte lines) and writes its digits straight into the
// planes, one 16-byte store per plane.
template <class Src>
__device__ __forceinline__ void planes_b_kmajor(const Src& src, __nv_bfloat16* out, i64 N, i64 K,
                                                i64 Kp, int bx, int by) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const i64 t = (i64)bx * 8 + w;
  const i64 n = (i64)by * 16 + (l >> 1);
  if (t >= Kp / KS || n >= N) return;
  const i64 k0 = t * KS + (l & 1) * 8;
  u64 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = k0 + e < K ? src((k0 + e) * N + n) : 0ull;
  write_planes(v, out, n, Kp, k0);
}

// B side of a convolution, gathered straight from the data (implicit im2col),
// K-major: lane l of warp w owns output column n = 16 by + l / 2 and the 8
// consecutive k of half l % 2 of sub-step t = 8 bx + w, so that it writes its
// digits straight into the planes ([n][Kp / 16][8][16]: one 16-byte store per
// plane, the lane pair filling whole 32-byte sectors) with no shared-memory
// transpose, and the 16 columns of a warp read 16 consecutive data positions
// per k.  Output z: z = 0 is pair 1, the opened sum over src1 - sub1 (shared
// by all jobs), written to outs.j[0]; z = 1 + j is job j's pair 2, src2[j],
// written to outs.j[1 + j].  Each output has blocks of its own: one gather
// feeding all of them (80 registers for three) ran at half the occupancy and
// made the speech step 2 % slower.
__device__ __forceinline__ void planes_b_conv_kmajor(const ConvGather& cg, const PlaneJobs& outs,
                                                     int N, int K, int Kp, int bx, int by, int z) {
  const mpc_conv_desc& d = cg.d;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int t = bx * 8 + w;
  const int n = by * 16 + (l >> 1);
  if (t >= Kp / KS || n >= N) return;
  const int k0 = t * KS + (l & 1) * 8;
  const int H = (int)d.h, W = (int)d.w, kh = (int)d.kh, kw = (int)d.kw;
  // Output column n -> (b, oh, ow) and the data offset of its window origin
  // (32-bit: the host checks that every data offset fits).
  const int wo = (int)cg.wo, ho = (int)cg.ho;
  const int ow = n % wo, tq = n / wo, oh = tq % ho, b = tq / ho;
  const int oy = oh * (int)d.stride_h - (int)d.pad_h, ox = ow * (int)d.stride_w - (int)d.pad_w;
  const int base = (b * (int)d.c_in * H + oy) * W + ox;
  // Tap (ci, r, s) of k0, advanced per k.
  const int khw = kh * kw;
  int ci = k0 / khw;
  int r = (k0 - ci * khw) / kw;
  int sx = k0 - ci * khw - r * kw;
  const u64* src2 = z > 0 ? cg.src2[z - 1] : nullptr;
  u64 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int y = oy + r, x = ox + sx;
    v[e] = 0;
    if (k0 + e < K && (unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W) {
      const int off = base + (ci * H + r) * W + sx;
      if (z == 0) {
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
    if (++sx == kw) {
      sx = 0;
      if (++r == kh) {
        r = 0;
        ++ci;
      }
    }
  }
  write_planes(v, outs.j[z].out, n, Kp, k0);
}

// One launch for both plane sides of a GEMM: blocks [0, na * a_blk) cut the A
// sources (a_blk blocks per job), the rest the B tiles (bx x by per source,
// nb sources), the B side either from row-major X or, with GATHER, from the
// convolution data.  Saves a kernel boundary per GEMM.
struct PlanesLaunch {
  PlaneJobs ja, jb;
  ConvGather cg;
  i64 M, N, K, Kp;
  int na, a_blk, nb, bx, by;
  int z0;  // B side: first output index (gather z0 .. z0 + nb - 1)
};

// B-side blocks cover 8 sub-steps x 16 columns (bx x by per source), from
// row-major X or, with GATHER, from the convolution data.
template <bool GATHER>
__global__ void __launch_bounds__(256) limb_planes(const __grid_constant__ PlanesLaunch pl) {
  const i64 b = blockIdx.x;
  const i64 a_blocks = (i64)pl.na * pl.a_blk;
  if (b < a_blocks) {
    const PlaneJob& jb = pl.ja.j[b / pl.a_blk];
    planes_a_part(DirectSrc{jb.X1}, jb.out, pl.M, pl.K, pl.Kp, b % pl.a_blk, pl.a_blk);
    return;
  }
  const int r = (int)(b - a_blocks);
  const int bx = r % pl.bx, by = (r / pl.bx) % pl.by, z = pl.z0 + r / (pl.bx * pl.by);
  if (GATHER)
    planes_b_conv_kmajor(pl.cg, pl.jb, (int)pl.N, (int)pl.K, (int)pl.Kp, bx, by, z);
  else
    planes_b_kmajor(DirectSrc{pl.jb.j[z].X1}, pl.jb.j[z].out, pl.N, pl.K, pl.Kp,
                    bx, by);
}

// The digit planes of many products in one launch (limb_planes_grouped): a
// task is one side of one product, block b belongs to the last task whose
// block_base <= b.
//
// A side of a Beaver product, from one read of X and A: the opened
// E = sum_p (X_p - A_p) and every party's A_p, each cut into digit planes
// ([M][K] row-major sources, parties pstride words apart); E's planes go to
// out, A_p's to out + (1 + p) ostride.  Block `blk` of `nblk` strides over the
// 8-k groups.
__device__ __forceinline__ void planes_a_beaver(const u64* __restrict__ X,
                                                const u64* __restrict__ S, i64 pstride, int P,
                                                __nv_bfloat16* out, i64 ostride, i64 M, i64 K,
                                                i64 Kp, i64 blk, i64 nblk) {
  const i64 kc = Kp / 8;
  const i64 total = M * kc;
  for (i64 i = blk * (i64)blockDim.x + threadIdx.x; i < total; i += nblk * blockDim.x) {
    const i64 m = i / kc, k0 = (i % kc) * 8;
    u64 e[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) e[j] = 0;
    for (int p = 0; p < P; ++p) {
      u64 a[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const i64 k = k0 + j;
        a[j] = 0;
        if (k < K) {
          const i64 idx = p * pstride + m * K + k;
          a[j] = S[idx];
          e[j] += X[idx] - a[j];
        }
      }
      write_planes(a, out + (1 + p) * ostride, m, Kp, k0);
    }
    write_planes(e, out, m, Kp, k0);
  }
}

// B side of a Beaver product, K-major like planes_b_kmajor, from one read of
// Y and B: F = sum_p (Y_p - B_p), G = B_0 + F and B_1 .. B_{P-1} ([K][N]
// row-major sources, parties pstride words apart); G's planes go to out, B_p's
// to out + p ostride, F's to out + P ostride.
__device__ __forceinline__ void planes_b_beaver(const u64* __restrict__ Y,
                                                const u64* __restrict__ S, i64 pstride, int P,
                                                __nv_bfloat16* out, i64 ostride, i64 N, i64 K,
                                                i64 Kp, int bx, int by) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const i64 t = (i64)bx * 8 + w;
  const i64 n = (i64)by * 16 + (l >> 1);
  if (t >= Kp / KS || n >= N) return;
  const i64 k0 = t * KS + (l & 1) * 8;
  u64 f[8], b0[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) f[j] = 0;
  for (int p = 0; p < P; ++p) {
    u64 b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      b[j] = 0;
      if (k0 + j < K) {
        const i64 idx = p * pstride + (k0 + j) * N + n;
        b[j] = S[idx];
        f[j] += Y[idx] - b[j];
      }
    }
    if (p == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) b0[j] = b[j];
    } else {
      write_planes(b, out + p * ostride, n, Kp, k0);
    }
  }
  write_planes(f, out + P * ostride, n, Kp, k0);
#pragma unroll
  for (int j = 0; j < 8; ++j) f[j] += b0[j];
  write_planes(f, out, n, Kp, k0);
}

// One side of one product of a grouped launch: the planes of its P + 1
// sources (side 0: E, A_0 .. A_{P-1}; side 1: G, B_1 .. B_{P-1}, F), which
// sit ostride bf16 apart from out in map order.
struct __align__(16) PlaneTask {
  const u64* src;  // X or Y
  const u64* sub;  // A or B
  __nv_bfloat16* out;
  i64 ostride;
  i64 rows, K, Kp;
  i64 block_base;
  i64 pstride;
  int side;  // 0: A side, 1: B side (transposed)
  int nblk;  // blocks of this task
  int bx;    // B side: tiles of 8 sub-steps
  int P;
};

__global__ void __launch_bounds__(256, 3) limb_planes_grouped(const PlaneTask* __restrict__ tasks,
                                                           int ntasks) {
  const i64 b = blockIdx.x;
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].block_base <= b) lo = mid; else hi = mid - 1;
  }
  const PlaneTask& t = tasks[lo];
  const i64 local = b - t.block_base;
  if (t.side == 0)
    planes_a_beaver(t.src, t.sub, t.pstride, t.P, t.out, t.ostride, t.rows, t.K, t.Kp, local,
                    t.nblk);
  else
    planes_b_beaver(t.src, t.sub, t.pstride, t.P, t.out, t.ostride, t.rows, t.K, t.Kp,
                    (int)(local % t.bx), (int)(local / t.bx));
}

// Copies a block of kernel parameters to device memory: how the grouped
// launch's tables reach the device without a host-memory copy, so that the
// call can be captured in a CUDA graph (the bytes are baked into the graph).
constexpr int kBlobBytes = 24 * 1024;
struct Blob {
  uint4 w[kBlobBytes / 16];
};

__global__ void __launch_bounds__(256) blob_copy_kernel(const __grid_constant__ Blob blob, int nwords,
                                                        uint4* __restrict__ dst) {
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = blob.w[i];
}

// Diagnostic for the bounded-wait status path: one thread waits, through
// mbar_wait and the CTA abort flag exactly as the engine's roles do, for the
// first phase of an mbarrier that nothing ever arrives at; the wait gives up
// after limit_ns and the CTA records MPC_ETIMEOUT the way limb_gemm_kernel does
// on an abort.  No copy, MMA or TMEM allocation is ever outstanding here, so
// the timeout path can be run on a GPU without any risk to the context.
__global__ void __launch_bounds__(32) wait_timeout_kernel(int* status,
                                                          unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t never_bar;
  __shared__ volatile int never_abort;
  if (threadIdx.x == 0) {
    mbar_init(&never_bar, 1);
    never_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0 && !mbar_wait(&never_bar, 0u, &never_abort, limit_ns))
    record_status(status, MPC_ETIMEOUT);
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

// 4-D map over interleaved planes [rows][Kp / 16][2][64] bf16 (the last two
// dims: planes 0..3 | 4..7 of a sub-step, 4 x 16 digits each) with a box of
// {64, 1, 1, box_rows}: 128 rows of 128 bytes, 128-byte swizzle.
int encode_planes(CUtensorMap* tm, const void* base, i64 rows, i64 Kp, int box_rows) {
  cuuint64_t dims[4] = {64, 2, (cuuint64_t)(Kp / KS), (cuuint64_t)rows};
  cuuint64_t strides[3] = {128, 256, (cuuint64_t)(Kp / KS) * 256};
  cuuint32_t box[4] = {64, 1, 1, (cuuint32_t)box_rows};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? MPC_OK : fail(MPC_ECUDA, "tensor map encode failed (%d)", (int)r);
}

// K of one operand pair rounded up to whole sub-steps.
inline i64 pair_k(i64 K) { return ceil_div(K, KS) * KS; }

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int limb_splits(i64 M, i64 N, i64 K, int npairs, int njobs, bool batch) {
  const i64 tiles = ceil_div(M, BM) * ceil_div(N, BN) * njobs;
  // A batch of one-pair products (the dealer's triples of same-shaped layers,
  // dealt on a low-priority stream beside the online phase) takes splits of
  // at least 32 sub-steps: for the speech dealer's six products that is 3
  // splits (252 CTAs of 38 sub-steps) instead of 7 (588 CTAs of 16), which
  // spends less of each CTA on its fixed set-up, fill and epilogue: the
  // dealer alone 6 % faster and the overlapped step 1 % faster.
  const i64 min_units = batch ? 32 : 16;
  return choose_splits(tiles, npairs * pair_k(K) / KS, min_units);
}

bool limb_supported(i64 M, i64 N, i64 K) {
  // TMA coordinates are 32-bit; keep every extent comfortably inside.
  return M >= 1 && N >= 1 && K >= 1 && M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 30);
}

size_t limb_workspace_bytes(i64 M, i64 N, i64 K, int npairs, int njobs) {
  // Upper bound: no pair shared between jobs.
  const i64 K1p = pair_k(K);
  return (size_t)njobs * npairs * (al256((size_t)8 * M * K1p * 2) + al256((size_t)8 * N * K1p * 2));
}

size_t limb_conv_prep_bytes(int P, i64 M, i64 N, i64 K) {
  const i64 K1p = pair_k(K);
  return (size_t)(P + 1) * al256((size_t)16 * M * K1p) + (size_t)P * al256((size_t)16 * N * K1p);
}

int limb_conv_prepare(int P, const ConvGather& cg, i64 M, i64 N, i64 K,
                      const u64* const* asrc, void* prep, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return MPC_OK;
  const i64 K1p = pair_k(K);
  const size_t a_bytes = al256((size_t)16 * M * K1p), b_bytes = al256((size_t)16 * N * K1p);
  char* w = static_cast<char*>(prep);
  const mpc_conv_desc& d = cg.d;
  const i64 data = d.batch * d.c_in * d.h * d.w;
  if (data >= (1ll << 31) || N >= (1ll << 31) || K1p >= (1ll << 31) ||
      (i64)8 * N * K1p >= (1ll << 62))
    return fail(MPC_EUNSUPPORTED, "convolution too large for the 32-bit gather");
  // One launch: A side the P + 1 weight-side sources in order, B side the
  // gather outputs 1 .. P (im2col(A_p)).
  KernelTimer timer("limb_planes", s);
  PlanesLaunch pl;
  memset(&pl, 0, sizeof(pl));
  pl.cg = cg;
  for (int j = 0; j <= P; ++j)
    pl.ja.j[j] = PlaneJob{asrc[j], nullptr,
                          reinterpret_cast<__nv_bfloat16*>(w + (size_t)j * a_bytes)};
  for (int p = 0; p < P; ++p)
    pl.jb.j[1 + p] = PlaneJob{nullptr, nullptr,
                              reinterpret_cast<__nv_bfloat16*>(w + (size_t)(P + 1) * a_bytes +
                                                               (size_t)p * b_bytes)};
  pl.M = M;
  pl.N = N;
  pl.K = K;
  pl.Kp = K1p;
  pl.na = P + 1;
  pl.a_blk = (int)std::min<i64>(ceil_div(M * (K1p / 8), 256), 148 * 4);
  pl.nb = P;
  pl.z0 = 1;
  pl.bx = (int)ceil_div(K1p / KS, 8);
  pl.by = (int)ceil_div(N, 16);
  const i64 blocks = (i64)pl.na * pl.a_blk + (i64)P * pl.bx * pl.by;
  if (blocks > 0x7FFFFFFFll) return fail(MPC_EUNSUPPORTED, "plane pass grid too large");
  limb_planes<true><<<(unsigned)blocks, 256, 0, s>>>(pl);
  return check_launch("limb_planes");
}

size_t limb_planes_a_bytes(i64 M, i64 K) { return al256((size_t)16 * M * pair_k(K)); }

int limb_cut_planes_a(int n, const u64* const* src, i64 M, i64 K, void* out, cudaStream_t s) {
  if (n <= 0 || M <= 0 || K <= 0) return MPC_OK;
  if (n > 2 * MPC_MAX_PARTIES) return fail(MPC_EINVAL, "too many plane sources");
  const i64 K1p = pair_k(K);
  const size_t bytes = limb_planes_a_bytes(M, K);
  KernelTimer timer("limb_planes", s);
  PlanesLaunch pl;
  memset(&pl, 0, sizeof(pl));
  for (int i = 0; i < n; ++i)
    pl.ja.j[i] = PlaneJob{src[i], nullptr,
                          reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(out) + i * bytes)};
  pl.M = M;
  pl.N = 1;
  pl.K = K;
  pl.Kp = K1p;
  pl.na = n;
  pl.nb = 0;
  pl.bx = pl.by = 1;
  pl.a_blk = (int)std::min<i64>(ceil_div(M * (K1p / 8), 256), 148 * 4);
  const i64 blocks = (i64)n * pl.a_blk;
  limb_planes<false><<<(unsigned)blocks, 256, 0, s>>>(pl);
  return check_launch("limb_planes");
}

int launch_gemm_limb(const GemmArgs& g_in, void* ws, size_t ws_bytes, cudaStream_t s) {
  GemmArgs g = g_in;
  if (g.splits < 1) g.splits = 1;
  if (g.M <= 0 || g.N <= 0 || g.njobs <= 0) return MPC_OK;
  if ((g.splits > 1 && g.partial == nullptr) || g.splits * g.njobs > 65535)
    return fail(MPC_EINVAL, "bad split configuration");
  if (!limb_supported(g.M, g.N, g.K)) return fail(MPC_EUNSUPPORTED, "shape outside limb engine");
  if (int rc = get_encoder()) return rc;
  const bool prep = g.prep != nullptr;
  if (prep && g.gather == nullptr)
    return fail(MPC_EINVAL, "limb engine: prepared planes need the convolution gather");
  const bool prep1 = prep && g.prep_pairs == 1;  // prepared products: one pair per job
  const int npairs = ((prep && !prep1) || (!prep && g.jobs[0].A2)) ? 2 : 1;
  const bool per_job = g.gather != nullptr && g.gather_per_job != 0;
  if (per_job && (npairs != 1 || prep))
    return fail(MPC_EINVAL, "limb engine: per-job gathers take one-pair products");
  for (int j = 1; j < g.njobs && !prep; ++j)
    if ((g.jobs[j].A2 != nullptr) != (npairs == 2))
      return fail(MPC_EINVAL, "limb engine: jobs mix one- and two-pair products");
  const i64 K1p = pair_k(g.K);
  const size_t need = limb_workspace_bytes(g.M, g.N, g.K, npairs, g.njobs);
  if (ws == nullptr || ws_bytes < need)
    return fail(MPC_ENOMEM, "limb workspace %zu bytes, need %zu", ws_bytes, need);
  const i64 gy = ceil_div(g.M, BM), gx = ceil_div(g.N, BN);
  if (gy > 65535) return fail(MPC_EUNSUPPORTED, "M too large for the limb engine grid");
  if (ceil_div(g.N, 16) > 0x7FFFFFFFll) return fail(MPC_EUNSUPPORTED, "N too large for the plane pass");
  int* st = device_status_ptr();
  if (!st) return fail(MPC_ECUDA, "device status word unavailable");

  // One plane buffer per distinct (side, pair, source); jobs that share a
  // source share its buffer and tensor map.
  LimbParams prm;
  memset(&prm, 0, sizeof(prm));
  char* w = static_cast<char*>(ws);
  const size_t a_bytes = al256((size_t)8 * g.M * K1p * 2), b_bytes = al256((size_t)8 * g.N * K1p * 2);
  PlaneJobs ja = {}, jbv = {};
  int na = 0, nb = 0;
  // Prepared planes (limb_conv_prepare): G, B_1 .. B_{P-1}, F, then im2col(A_p).
  const char* pp = static_cast<const char*>(g.prep);
  if (prep) {
    for (int j = 0; j < g.njobs; ++j) {
      if (int rc = encode_planes(&prm.tmA[0][j], pp + (size_t)j * a_bytes, g.M, K1p, BM)) return rc;
      if (prep1) continue;
      if (int rc = encode_planes(&prm.tmA[1][j], pp + (size_t)g.njobs * a_bytes, g.M, K1p, BM))
        return rc;
    }
  }
  for (int pr = 0; pr < npairs && !prep && !per_job; ++pr) {
    for (int j = 0; j < g.njobs; ++j) {
      const u64* src = pr ? g.jobs[j].A2 : g.jobs[j].A1;
      int hit = -1;
      for (int u = 0; u < na; ++u)
        if (ja.j[u].X1 == src) hit = u;
      if (hit < 0) {
        ja.j[na] = PlaneJob{src, nullptr, reinterpret_cast<__nv_bfloat16*>(w)};
        w += a_bytes;
        hit = na++;
      }
      if (int rc = encode_planes(&prm.tmA[pr][j], ja.j[hit].out, g.M, K1p, BM)) return rc;
    }
  }
  if (per_job) {
    // Job j is its own convolution g.gather[j] (same M and N for all jobs, K_j
    // <= g.K): planes A_j (M x K_j) of jobs[j].A1 and B_j (N x K_j) gathered
    // from g.gather[j].src2[0], its own sub-step count Tj[j]; one plane launch
    // per run of jobs with one descriptor.
    KernelTimer timer("limb_planes", s);
    for (int j0 = 0; j0 < g.njobs;) {
      const ConvGather& c0 = g.gather[j0];
      int j1 = j0 + 1;
      while (j1 < g.njobs && memcmp(&g.gather[j1].d, &c0.d, sizeof(c0.d)) == 0) ++j1;
      const i64 Kj = c0.d.c_in * c0.d.kh * c0.d.kw, Kjp = pair_k(Kj);
      const i64 data = c0.d.batch * c0.d.c_in * c0.d.h * c0.d.w;
      if (Kj < 1 || Kj > g.K || data >= (1ll << 31) || (i64)8 * g.N * Kjp >= (1ll << 62))
        return fail(MPC_EUNSUPPORTED, "per-job convolution outside the limb gather");
      if (Kjp / KS < g.splits) return fail(MPC_EUNSUPPORTED, "per-job K shorter than its splits");
      PlanesLaunch pl;
      memset(&pl, 0, sizeof(pl));
      pl.cg = c0;
      pl.M = g.M;
      pl.N = g.N;
      pl.K = Kj;
      pl.Kp = Kjp;
      pl.na = pl.nb = j1 - j0;
      pl.z0 = 1;
      for (int j = j0; j < j1; ++j) {
        const int i = j - j0;
        pl.ja.j[i] = PlaneJob{g.jobs[j].A1, nullptr, reinterpret_cast<__nv_bfloat16*>(w)};
        if (int rc = encode_planes(&prm.tmA[0][j], w, g.M, Kjp, BM)) return rc;
        w += al256((size_t)16 * g.M * Kjp);
        pl.jb.j[1 + i] = PlaneJob{nullptr, nullptr, reinterpret_cast<__nv_bfloat16*>(w)};
        if (int rc = encode_planes(&prm.tmB[0][j], w, g.N, Kjp, BN)) return rc;
        w += al256((size_t)16 * g.N * Kjp);
        pl.cg.src2[i] = g.gather[j].src2[0];
        prm.Tj[j] = (int)(Kjp / KS);
      }
      pl.bx = (int)ceil_div(Kjp / KS, 8);
      pl.by = (int)ceil_div(g.N, 16);
      pl.a_blk = (int)std::min<i64>(ceil_div(g.M * (Kjp / 8), 256), 148 * 4);
      const i64 blocks = (i64)pl.na * pl.a_blk + (i64)pl.nb * pl.bx * pl.by;
      if (blocks > 0x7FFFFFFFll) return fail(MPC_EUNSUPPORTED, "plane pass grid too large");
      limb_planes<true><<<(unsigned)blocks, 256, 0, s>>>(pl);
      if (int rc = check_launch("limb_planes")) return rc;
      j0 = j1;
    }
  } else if (g.gather) {
    // pair 1: the opened gather, shared; pair 2 (two-pair products): one per job
    nb = (npairs == 2 && !prep) ? 1 + g.njobs : 1;
    for (int z = 0; z < nb; ++z) {
      jbv.j[z] = PlaneJob{nullptr, nullptr, reinterpret_cast<__nv_bfloat16*>(w)};
      w += b_bytes;
    }
    for (int j = 0; j < g.njobs; ++j) {
      if (int rc = encode_planes(&prm.tmB[0][j], jbv.j[0].out, g.N, K1p, BN)) return rc;
      if (prep && !prep1) {
        const char* bj = pp + (size_t)(g.njobs + 1) * a_bytes + (size_t)j * b_bytes;
        if (int rc = encode_planes(&prm.tmB[1][j], bj, g.N, K1p, BN)) return rc;
      } else if (npairs == 2) {
        if (int rc = encode_planes(&prm.tmB[1][j], jbv.j[1 + j].out, g.N, K1p, BN)) return rc;
      }
    }
  } else {
    for (int pr = 0; pr < npairs; ++pr) {
      for (int j = 0; j < g.njobs; ++j) {
        const u64* src = pr ? g.jobs[j].B2 : g.jobs[j].B1;
        int hit = -1;
        for (int u = 0; u < nb; ++u)
          if (jbv.j[u].X1 == src) hit = u;
        if (hit < 0) {
          jbv.j[nb] = PlaneJob{src, nullptr, reinterpret_cast<__nv_bfloat16*>(w)};
          w += b_bytes;
          hit = nb++;
        }
        if (int rc = encode_planes(&prm.tmB[pr][j], jbv.j[hit].out, g.N, K1p, BN)) return rc;
      }
    }
  }
  for (int j = 0; j < g.njobs; ++j) {
    prm.C[j] = g.jobs[j].C;
    prm.Z[j] = g.jobs[j].Z;
  }
  if (!per_job) {
    KernelTimer timer("limb_planes", s);
    PlanesLaunch pl;
    memset(&pl, 0, sizeof(pl));
    pl.ja = ja;
    pl.jb = jbv;
    pl.M = g.M;
    pl.N = g.N;
    pl.K = g.K;
    pl.Kp = K1p;
    pl.na = na;
    pl.nb = nb;
    pl.bx = (int)ceil_div(K1p / KS, 8);  // B side: blocks of 8 sub-steps x 16 columns
    pl.by = (int)ceil_div(g.N, 16);
    // A side: about as many threads as 8-k groups, at most 4 blocks per SM and job.
    pl.a_blk = (int)std::min<i64>(ceil_div(g.M * (K1p / 8), 256), 148 * 4);
    const i64 blocks = (i64)na * pl.a_blk + (i64)nb * pl.bx * pl.by;
    if (blocks > 0x7FFFFFFFll) return fail(MPC_EUNSUPPORTED, "plane pass grid too large");
    if (g.gather) {
      const mpc_conv_desc& d = g.gather->d;
      const i64 data = d.batch * d.c_in * d.h * d.w;
      if (data >= (1ll << 31) || g.N >= (1ll << 31) || K1p >= (1ll << 31) ||
          (i64)8 * g.N * K1p >= (1ll << 62))
        return fail(MPC_EUNSUPPORTED, "convolution too large for the 32-bit gather");
      pl.cg = *g.gather;
      limb_planes<true><<<(unsigned)blocks, 256, 0, s>>>(pl);
    } else {
      limb_planes<false><<<(unsigned)blocks, 256, 0, s>>>(pl);
    }
    if (int rc = check_launch("limb_planes")) return rc;
  }
  prm.M = g.M;
  prm.N = g.N;
  prm.hw_out = g.hw_out;
  prm.T1 = (int)(K1p / KS);
  prm.T = npairs * prm.T1;
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
  return (g.splits > 1 && !g.defer_reduce) ? gemm_reduce(g, s) : MPC_OK;
}

namespace {

// Workspace of a grouped launch, each region 256-byte aligned: the work
// counter, the product table, the tensor maps (2 (P + 1) per product), the
// plane tasks, then every product's digit planes (A side 1 + P sources of
// M x K1p, B side P + 1 sources of N x K1p, 16 bytes per word).
struct GroupLayout {
  size_t prods_off, maps_off, tasks_off, planes_off, total;
};

GroupLayout group_layout(int P, int count, const GroupedProduct* prods) {
  GroupLayout L;
  size_t off = 256;
  L.prods_off = off;
  off += al256((size_t)count * sizeof(GroupProd));
  L.maps_off = off;
  off += al256((size_t)count * 2 * (P + 1) * sizeof(CUtensorMap));
  L.tasks_off = off;
  off += al256((size_t)count * 2 * (P + 1) * sizeof(PlaneTask));
  L.planes_off = off;
  for (int i = 0; i < count; ++i) {
    const i64 K1p = pair_k(prods[i].K);
    off += (size_t)(P + 1) * (al256((size_t)16 * prods[i].M * K1p) +
                              al256((size_t)16 * prods[i].N * K1p));
  }
  L.total = off;
  return L;
}

// Copies `bytes` (a multiple of 16) from host memory to the device through
// kernel parameters, kBlobBytes per launch.
int upload_params(const void* src, size_t bytes, void* dst, cudaStream_t s) {
  const uint8_t* p = static_cast<const uint8_t*>(src);
  uint8_t* d = static_cast<uint8_t*>(dst);
  for (size_t off = 0; off < bytes; off += kBlobBytes) {
    const size_t n = std::min<size_t>(kBlobBytes, bytes - off);
    Blob blob;
    memcpy(&blob, p + off, n);
    blob_copy_kernel<<<1, 256, 0, s>>>(blob, (int)(n / 16), reinterpret_cast<uint4*>(d + off));
    if (int rc = check_launch("table upload")) return rc;
  }
  return MPC_OK;
}

}  // namespace

size_t limb_grouped_workspace_bytes(int P, int count, const GroupedProduct* prods) {
  return group_layout(P, count, prods).total;
}

int launch_gemm_limb_grouped(int P, int count, const GroupedProduct* prods, int trunc_bits,
                             int ctas, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (count <= 0) return MPC_OK;
  if (int rc = get_encoder()) return rc;
  for (int i = 0; i < count; ++i)
    if (!limb_supported(prods[i].M, prods[i].N, prods[i].K))
      return fail(MPC_EUNSUPPORTED, "grouped limb product %d outside the limb engine", i);
  const GroupLayout L = group_layout(P, count, prods);
  if (ws == nullptr || ws_bytes < L.total)
    return fail(MPC_ENOMEM, "grouped limb workspace %zu bytes, need %zu", ws_bytes, L.total);
  int* st = device_status_ptr();
  if (!st) return fail(MPC_ECUDA, "device status word unavailable");
  char* base = static_cast<char*>(ws);
  GroupProd* d_prods = reinterpret_cast<GroupProd*>(base + L.prods_off);
  CUtensorMap* d_maps = reinterpret_cast<CUtensorMap*>(base + L.maps_off);
  PlaneTask* d_tasks = reinterpret_cast<PlaneTask*>(base + L.tasks_off);

  const int nmaps = 2 * (P + 1);
  std::vector<GroupProd> hp(count);
  std::vector<CUtensorMap> hm((size_t)count * nmaps);
  std::vector<PlaneTask> ht;
  ht.reserve((size_t)count * nmaps);
  char* planes = base + L.planes_off;
  i64 tile_base = 0, block_base = 0;
  for (int i = 0; i < count; ++i) {
    const GroupedProduct& g = prods[i];
    const i64 K1p = pair_k(g.K);
    const size_t a_bytes = al256((size_t)16 * g.M * K1p), b_bytes = al256((size_t)16 * g.N * K1p);
    // Sources in map order: A side E, A_0..A_{P-1}; B side G, B_1..B_{P-1},
    // F, each side's planes consecutive.  One task per side cuts all of them
    // from one read of the shares (E = sum_p (X_p - A_p) and
    // F = sum_p (Y_p - B_p) are opened inside the pass, G = B_0 + F).
    const i64 mk = g.M * g.K, kn = g.K * g.N;
    for (int side = 0; side < 2; ++side) {
      const bool aside = side == 0;
      const i64 rows = aside ? g.M : g.N;
      const size_t bytes = aside ? a_bytes : b_bytes;
      __nv_bfloat16* first = reinterpret_cast<__nv_bfloat16*>(planes);
      for (int j = 0; j <= P; ++j) {
        const int m = aside ? j : P + 1 + j;
        if (int rc = encode_planes(&hm[(size_t)i * nmaps + m], planes, rows, K1p, aside ? BM : BN))
          return rc;
        planes += bytes;
      }
      PlaneTask t{};
      t.src = aside ? g.X : g.Y;
      t.sub = aside ? g.A : g.B;
      t.pstride = aside ? mk : kn;
      t.P = P;
      t.out = first;
      t.ostride = (i64)(bytes / sizeof(__nv_bfloat16));
      t.rows = rows;
      t.K = g.K;
      t.Kp = K1p;
      t.block_base = block_base;
      t.side = side;
      if (aside) {
        t.nblk = (int)std::min<i64>(ceil_div(g.M * (K1p / 8), 256), 148 * 4);
      } else {  // blocks of 8 sub-steps x 16 columns
        t.bx = (int)ceil_div(K1p / KS, 8);
        t.nblk = t.bx * (int)ceil_div(g.N, 16);
      }
      block_base += t.nblk;
      ht.push_back(t);
    }
    GroupProd& b = hp[i];
    b.M = g.M;
    b.N = g.N;
    b.tiles_m = (int)ceil_div(g.M, BM);
    b.tiles_n = (int)ceil_div(g.N, BN);
    b.tile_base = tile_base;
    tile_base += (i64)P * b.tiles_m * b.tiles_n;
    b.T1 = (int)(K1p / KS);
    b.P = P;
    b.C = g.C;
    b.Z = g.Z;
    b.maps = d_maps + (size_t)i * nmaps;
  }
  if (block_base > 0x7FFFFFFFll) return fail(MPC_EUNSUPPORTED, "grouped plane pass too large");
  static_assert(sizeof(GroupProd) % 16 == 0 && sizeof(PlaneTask) % 16 == 0, "16-byte records");
  if (int rc = upload_params(hp.data(), hp.size() * sizeof(GroupProd), d_prods, s)) return rc;
  if (int rc = upload_params(hm.data(), hm.size() * sizeof(CUtensorMap), d_maps, s)) return rc;
  if (int rc = upload_params(ht.data(), ht.size() * sizeof(PlaneTask), d_tasks, s)) return rc;
  {
    KernelTimer timer("limb_planes", s);
    limb_planes_grouped<<<(unsigned)block_base, 256, 0, s>>>(d_tasks, (int)ht.size());
    if (int rc = check_launch("limb_planes_grouped")) return rc;
  }
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(MPC_ECUDA, "counter reset: %s", cudaGetErrorString(e));
  e = cudaFuncSetAttribute(limb_gemm_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_BYTES);
  if (e != cudaSuccess) return fail(MPC_ECUDA, "smem attribute: %s", cudaGetErrorString(e));
  GroupParams gp;
  gp.prods = d_prods;
  gp.count = count;
  gp.total = tile_base;
  gp.counter = counter;
  gp.trunc_bits = trunc_bits;
  gp.status = st;
  int dev = 0, sms = kPlanSMs;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const i64 grid = std::min<i64>(ctas > 0 ? ctas : sms, tile_base);
  {
    KernelTimer timer("gemm_limb", s);
    limb_gemm_grouped_kernel<<<(unsigned)grid, kThreads, SMEM_BYTES, s>>>(gp);
    if (int rc = check_launch("gemm_limb_grouped")) return rc;
  }
  return MPC_OK;
}

}  // namespace mpc

extern "C" int mpc_test_wait_timeout(int64_t limit_ns, void* stream) {
  using namespace mpc;
  MPC_REQUIRE(limit_ns >= 1000 && limit_ns <= 1000000000ll,
              "limit_ns %lld outside [1 us, 1 s]", (long long)limit_ns);
  int* st = device_status_ptr();
  if (!st) return fail(MPC_ECUDA, "device status word unavailable");
  wait_timeout_kernel<<<1, 32, 0, as_stream(stream)>>>(st, (unsigned long long)limit_ns);
  return check_launch("wait_timeout");
}
