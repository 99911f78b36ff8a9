// Function approximations on two-party shares (App. D.2), fused: one element
// per thread, the dealer's material regenerated from Philox in registers, every
// opening a sum over the two shares the thread holds.  A function of many
// interactive steps (exp: 8 squarings; reciprocal: exp plus 20 products) is one
// launch that reads x and writes the result, 32 bytes per element.
//
// Step k of a function draws its material at op id op + 10 k, in the order the
// steps run (a comparison uses op .. op + 3 of its block).  Fixed point 2^16;
// products of two scaled values are truncated by 16 bits, products with an
// unscaled 0/1 or +-1 sharing are not.
//
//   exp         limit approximation (1 + x / 2^n)^(2^n): truncate by n, n squarings
//   reciprocal  Newton-Raphson y <- y (2 - x y) from y0 = 3 exp(0.5 - x) + 0.003;
//               for either sign 1/x = sgn(x) / |x|, sgn(x) = 1 - 2 [x < 0]
//   sigmoid     sigma(|x|) by Newton-Raphson on 1 + exp(-|x|) from y0 = 0.75,
//               then [x < 0] ? 1 - sigma(|x|) : sigma(|x|) by one multiplexing product
//   tanh        2 sigma(2x) - 1
//   erf         Maclaurin series, odd powers by products with x^2
//   inv_sqrt    y <- y (3 - x y^2) / 2 from y0 = 3 g^16 + 0.3 g + 0.05, g = exp(-x/16)
//   log         Householder: h = 1 - x exp(-y), y <- y - sum_{k<=order} h^k / k,
//               from y0 = x / 120 - 20 exp(-2x - 1) + 3
//   max         tree of max(a, b) = b + ReLU(a - b) over adjacent pairs of the last axis
//   softmax     exp(x - max) * reciprocal(sum exp(x - max)), positive reciprocal
#include <cmath>

#include "common.cuh"
#include "fused.cuh"
#include "host.hpp"

namespace mpc {
namespace {

constexpr int kThreads = 256;
constexpr int kFrac = 16;
constexpr u64 kOne = 1ull << kFrac;
constexpr int kMaxCoef = 17;

enum Fn { kExp, kRecipPos, kRecip, kSigmoid, kTanh, kErf, kInvSqrt, kSqrt, kLog };

struct ApproxParams {
  int exp_iters;      // n of the limit approximation
  int nr_iters;       // Newton-Raphson iterations
  int terms;          // erf: K; log: polynomial order
  int log_iters;      // log: Householder iterations
  u64 c_recip_bias;   // enc(0.003)
  u64 c_sig_init;     // enc(0.75)
  u64 c_isq_bias;     // enc(0.05)
  u64 c_isq_g;        // enc(0.3)
  u64 c_log_lin;      // enc(1/120)
  u64 coef[kMaxCoef]; // erf: enc(2/sqrt(pi) (-1)^k / (k! (2k+1))); log: enc(1/k)
};

// rint(c 2^16), ties to even (the default rounding mode).
u64 enc(double c) { return (u64)(i64)std::nearbyint(c * (double)kOne); }

struct Ctx {
  u64 seed;
  i64 blk;
  int j;
};

__device__ __forceinline__ u64 neg(u64 v) { return 0ull - v; }

// ---- building blocks ------------------------------------------------------------------
__device__ __forceinline__ Sh2 d_exp(Sh2 x, int iters, const Ctx& c, u64& op) {
  Sh2 y = affine2(trunc2(x, iters), 1ull, kOne);  // 1 + x / 2^n
  for (int k = 0; k < iters; k += 4) {
    WordList<12> wl;
#pragma unroll
    for (int s = 0; s < 4; ++s) wl.add_square(op + 10ull * (k + s));
    wl.generate(c.seed, c.blk, c.j);
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (k + s < iters) y = sq2(y, wl.w + 3 * s, kFrac);
  }
  op += 10ull * iters;
  return y;
}

__device__ __forceinline__ Sh2 d_recip_nr(Sh2 x, Sh2 y, int iters, const Ctx& c, u64& op) {
  for (int k = 0; k < iters; k += 2) {
    WordList<20> wl;
#pragma unroll
    for (int s = 0; s < 4; ++s) wl.add_mul(op + 10ull * (2 * k + s));
    wl.generate(c.seed, c.blk, c.j);
#pragma unroll
    for (int it = 0; it < 2; ++it)
      if (k + it < iters) {
        const Sh2 t = mul2(x, y, wl.w + 10 * it, kFrac);
        y = mul2(y, affine2(t, neg(1), 2 * kOne), wl.w + 10 * it + 5, kFrac);
      }
  }
  op += 20ull * iters;
  return y;
}

__device__ __forceinline__ Sh2 d_recip_pos(Sh2 x, const ApproxParams& p, const Ctx& c, u64& op) {
  const Sh2 e = d_exp(affine2(x, neg(1), kOne / 2), p.exp_iters, c, op);
  return d_recip_nr(x, affine2(e, 3ull, p.c_recip_bias), p.nr_iters, c, op);
}

// One product at the next op id (its five words plus three unused).
__device__ __forceinline__ Sh2 d_mul_once(Sh2 x, Sh2 y, int trunc_bits, const Ctx& c, u64& op) {
  WordList<8> wl;
  wl.add_mul(op);
  wl.generate(c.seed, c.blk, c.j);
  op += 10;
  return mul2(x, y, wl.w, trunc_bits);
}

// [x < 0] (returned), sgn(x) = 1 - 2 [x < 0] and |x| = sgn(x) x: a comparison and
// one product; the product's c_0 rides in the comparison's spare slot.
__device__ __forceinline__ Sh2 d_sign_split(Sh2 x, const Ctx& c, u64& op, Sh2& sgn, Sh2& ax) {
  const u64 op_mul = op + 10;
  u64 w[5];
  const Sh2 bit = ltz_quad(x, c.seed, op, c.blk, c.j, op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_C, 0, 0), w[4]);
  const Quad4 t = quad_gen(c.seed, op_mul, stream_word2(MPC_ROLE_TRIPLE_A, 0, 0), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_A, 0, 1), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_B, 0, 0), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_B, 0, 1), c.blk, c.j);
#pragma unroll
  for (int s = 0; s < 4; ++s) w[s] = t.w[s];
  sgn = affine2(bit, neg(2), 1ull);
  ax = mul2(x, sgn, w, 0);
  op += 20;
  return bit;
}

__device__ __forceinline__ Sh2 d_sigmoid(Sh2 x, const ApproxParams& p, const Ctx& c, u64& op) {
  Sh2 sgn, ax;
  const Sh2 bit = d_sign_split(x, c, op, sgn, ax);
  const Sh2 d = affine2(d_exp(affine2(ax, neg(1), 0ull), p.exp_iters, c, op), 1ull, kOne);
  const Sh2 s = d_recip_nr(d, Sh2{{p.c_sig_init, 0ull}}, p.nr_iters, c, op);  // sigma(|x|)
  // multiplexing: [c] ((1 - s) - s) + s
  const Sh2 diff = sub2(affine2(s, neg(1), kOne), s);
  return add2(d_mul_once(bit, diff, 0, c, op), s);
}

__device__ __forceinline__ Sh2 d_erf(Sh2 x, const ApproxParams& p, const Ctx& c, u64& op) {
  const int K = p.terms;
  WordList<8> first;  // x^2, then the first product
  first.add_square(op);
  first.add_mul(op + 10);
  first.generate(c.seed, c.blk, c.j);
  const Sh2 x2 = sq2(x, first.w, kFrac);
  Sh2 acc = affine2(x, p.coef[0], 0ull, kFrac);
  Sh2 pw = x;
  if (K >= 1) {
    pw = mul2(pw, x2, first.w + 3, kFrac);
    acc = add2(acc, affine2(pw, p.coef[1], 0ull, kFrac));
  }
  for (int k = 2; k <= K; k += 4) {
    WordList<20> wl;
#pragma unroll
    for (int s = 0; s < 4; ++s) wl.add_mul(op + 10ull * (k + s));
    wl.generate(c.seed, c.blk, c.j);
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (k + s <= K) {
        pw = mul2(pw, x2, wl.w + 5 * s, kFrac);
        acc = add2(acc, affine2(pw, p.coef[k + s], 0ull, kFrac));
      }
  }
  op += 10ull * (K + 1);
  return acc;
}

__device__ __forceinline__ Sh2 d_inv_sqrt(Sh2 x, const ApproxParams& p, const Ctx& c, u64& op) {
  const Sh2 g = d_exp(affine2(x, neg(1), 0ull, 4), p.exp_iters, c, op);  // exp(-x / 16)
  WordList<12> sq;
#pragma unroll
  for (int s = 0; s < 4; ++s) sq.add_square(op + 10ull * s);
  sq.generate(c.seed, c.blk, c.j);
  Sh2 e = g;
#pragma unroll
  for (int s = 0; s < 4; ++s) e = sq2(e, sq.w + 3 * s, kFrac);  // exp(-x)
  op += 40;
  Sh2 y = add2(affine2(e, 3ull, p.c_isq_bias), affine2(g, p.c_isq_g, 0ull, kFrac));
  for (int it = 0; it < p.nr_iters; ++it) {
    WordList<16> wl;  // y^2, x y^2, y (3 - x y^2): 13 words
    wl.add_square(op);
    wl.add_mul(op + 10);
    wl.add_mul(op + 20);
    wl.generate(c.seed, c.blk, c.j);
    const Sh2 t = mul2(x, sq2(y, wl.w, kFrac), wl.w + 3, kFrac);
    y = mul2(y, affine2(t, neg(1), 3 * kOne), wl.w + 8, kFrac + 1);
    op += 30;
  }
  return y;
}

__device__ __forceinline__ Sh2 d_log(Sh2 x, const ApproxParams& p, const Ctx& c, u64& op) {
  const Sh2 lin = affine2(x, p.c_log_lin, 0ull, kFrac);
  const Sh2 e0 = d_exp(affine2(x, neg(2), neg(kOne)), p.exp_iters, c, op);
  Sh2 y = add2(lin, affine2(e0, neg(20), 3 * kOne));
  const int order = p.terms;
  for (int it = 0; it < p.log_iters; ++it) {
    const Sh2 em = d_exp(affine2(y, neg(1), 0ull), p.exp_iters, c, op);  // exp(-y)
    Sh2 h = em, pw = em, s = em;
    for (int m = 0; m < order; m += 4) {  // product m: x e^-y (m = 0), else h^(m+1)
      WordList<20> wl;
#pragma unroll
      for (int q = 0; q < 4; ++q) wl.add_mul(op + 10ull * (m + q));
      wl.generate(c.seed, c.blk, c.j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = m + q;
        if (k == 0) {
          h = affine2(mul2(x, em, wl.w, kFrac), neg(1), kOne);
          pw = h;
          s = h;
        } else if (k < order) {
          pw = mul2(pw, h, wl.w + 5 * q, kFrac);
          s = add2(s, affine2(pw, p.coef[k + 1], 0ull, kFrac));
        }
      }
    }
    op += 10ull * order;
    y = sub2(y, s);
  }
  return y;
}

template <int FN>
__device__ __forceinline__ Sh2 apply(Sh2 x, const ApproxParams& p, const Ctx& c, u64 op) {
  if (FN == kExp) return d_exp(x, p.exp_iters, c, op);
  if (FN == kRecipPos) return d_recip_pos(x, p, c, op);
  if (FN == kRecip) {
    Sh2 sgn, ax;
    d_sign_split(x, c, op, sgn, ax);
    const Sh2 r = d_recip_pos(ax, p, c, op);
    return d_mul_once(r, sgn, 0, c, op);
  }
  if (FN == kSigmoid) return d_sigmoid(x, p, c, op);
  if (FN == kTanh) return affine2(d_sigmoid(affine2(x, 2ull, 0ull), p, c, op), 2ull, neg(kOne));
  if (FN == kErf) return d_erf(x, p, c, op);
  if (FN == kInvSqrt) return d_inv_sqrt(x, p, c, op);
  if (FN == kSqrt) {
    const Sh2 r = d_inv_sqrt(x, p, c, op);
    return d_mul_once(x, r, kFrac, c, op);
  }
  return d_log(x, p, c, op);
}

// Shares [2][n]; Y may alias X.  Grid-stride with a uniform trip count per block
// so that every lane of a warp takes part in the quad shuffles.
template <int FN>
__global__ void __launch_bounds__(kThreads) approx_kernel(i64 n, const u64* X, u64* Y, u64 seed,
                                                          u64 op, const ApproxParams p) {
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(n, (i64)blockDim.x) * blockDim.x;
  const int j = threadIdx.x & 3;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < npad; i += stride) {
    const bool valid = i < n;
    const Sh2 x{{valid ? X[i] : 0ull, valid ? X[n + i] : 0ull}};
    const Sh2 y = apply<FN>(x, p, Ctx{seed, i >> 2, j}, op);
    if (valid) {
      Y[i] = y.v[0];
      Y[n + i] = y.v[1];
    }
  }
}

// One level of the max tree over the last axis: X [2][rows][m] -> O [2][rows][ceil(m/2)],
// O[r][i] = b + ReLU(a - b) for (a, b) = X[r][2i], X[r][2i+1]; the ReLU's material
// is indexed by the flat pair index r * floor(m/2) + i.  An odd last element is copied.
__global__ void __launch_bounds__(kThreads) max_level_kernel(i64 rows, i64 m, const u64* X,
                                                             u64* O, u64 seed, u64 op) {
  const i64 npairs = m / 2, mo = m - npairs;
  const i64 total = rows * npairs;
  const i64 in_stride = rows * m, out_stride = rows * mo;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(total, (i64)blockDim.x) * blockDim.x;
  const int j = threadIdx.x & 3;
  for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t - threadIdx.x < npad; t += stride) {
    const bool valid = t < total;
    const i64 r = valid ? t / npairs : 0, i = valid ? t - r * npairs : 0;
    const i64 src = r * m + 2 * i;
    Sh2 a{{0ull, 0ull}}, b{{0ull, 0ull}};
    if (valid) {
      a = Sh2{{X[src], X[in_stride + src]}};
      b = Sh2{{X[src + 1], X[in_stride + src + 1]}};
    }
    const Sh2 y = add2(b, relu_quad(sub2(a, b), seed, op, t >> 2, j));
    if (valid) {
      const i64 dst = r * mo + i;
      O[dst] = y.v[0];
      O[out_stride + dst] = y.v[1];
    }
  }
  if (m & 1) {
    for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
      O[r * mo + npairs] = X[r * m + m - 1];
      O[out_stride + r * mo + npairs] = X[in_stride + r * m + m - 1];
    }
  }
}

// E = exp(X - MX[row]) over [2][rows][m] (flat material index), and S[p][row] +=
// the row sums of E (S zeroed by the caller).  Ring addition is associative and
// commutative, so the atomic accumulation is exact and order-independent.
__global__ void __launch_bounds__(kThreads) softmax_exp_kernel(i64 rows, i64 m, const u64* X,
                                                               const u64* MX, u64* E, u64* S,
                                                               u64 seed, u64 op, int iters) {
  const i64 n = rows * m;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(n, (i64)blockDim.x) * blockDim.x;
  const int j = threadIdx.x & 3;
  const int lane = threadIdx.x & 31;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < npad; i += stride) {
    const bool valid = i < n;
    const i64 r = valid ? i / m : -1;
    Sh2 z{{0ull, 0ull}};
    if (valid) z = Sh2{{X[i] - MX[r], X[n + i] - MX[rows + r]}};
    u64 opk = op;
    Sh2 e = d_exp(z, iters, Ctx{seed, i >> 2, j}, opk);
    if (valid) {
      E[i] = e.v[0];
      E[n + i] = e.v[1];
    } else {
      e = Sh2{{0ull, 0ull}};
    }
    // segmented sum over the lanes of one row (rows are contiguous in i)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u64 u0 = __shfl_down_sync(0xffffffffu, e.v[0], d);
      const u64 u1 = __shfl_down_sync(0xffffffffu, e.v[1], d);
      const i64 ru = __shfl_down_sync(0xffffffffu, r, d);
      if (lane + d < 32 && ru == r) {
        e.v[0] += u0;
        e.v[1] += u1;
      }
    }
    const i64 rprev = __shfl_up_sync(0xffffffffu, r, 1);
    if (valid && (lane == 0 || rprev != r)) {
      atomicAdd((unsigned long long*)&S[r], (unsigned long long)e.v[0]);
      atomicAdd((unsigned long long*)&S[rows + r], (unsigned long long)e.v[1]);
    }
  }
}

// Y = trunc(E * R[row]) over [2][rows][m]: a Beaver product with the elementwise
// triple at op (flat index), R broadcast along the row.  Y may alias E.
__global__ void __launch_bounds__(kThreads) row_scale_kernel(i64 rows, i64 m, const u64* E,
                                                             const u64* R, u64* Y, u64 seed,
                                                             u64 op) {
  const i64 n = rows * m;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(n, (i64)blockDim.x) * blockDim.x;
  const int j = threadIdx.x & 3;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < npad; i += stride) {
    const bool valid = i < n;
    const i64 r = valid ? i / m : 0;
    Sh2 e{{0ull, 0ull}}, y{{0ull, 0ull}};
    if (valid) {
      e = Sh2{{E[i], E[n + i]}};
      y = Sh2{{R[r], R[rows + r]}};
    }
    u64 opk = op;
    const Sh2 z = d_mul_once(e, y, kFrac, Ctx{seed, i >> 2, j}, opk);
    if (valid) {
      Y[i] = z.v[0];
      Y[n + i] = z.v[1];
    }
  }
}

// ---- host side ------------------------------------------------------------------------
struct Cost {
  uint64_t rounds = 0, opened = 0, and_gates = 0, words = 0;
  void mul(uint64_t n, uint64_t k = 1) {
    rounds += k;
    opened += 16ull * n * k;
    words += 6ull * n * k;
  }
  void square(uint64_t n, uint64_t k = 1) {
    rounds += k;
    opened += 8ull * n * k;
    words += 4ull * n * k;
  }
  void ltz(uint64_t n) {
    rounds += 7 + 1;  // A2B: one AND round plus 6 prefix rounds; B2A: one
    opened += (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div((i64)n, 8);
    and_gates += (uint64_t)MPC_KS_GATES * n;
    words += (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n;
  }
  void relu(uint64_t n) {
    ltz(n);
    mul(n);
  }
};

ApproxParams make_params(int exp_iters, int nr_iters, int terms, int log_iters) {
  ApproxParams p{};
  p.exp_iters = exp_iters;
  p.nr_iters = nr_iters;
  p.terms = terms;
  p.log_iters = log_iters;
  p.c_recip_bias = enc(0.003);
  p.c_sig_init = enc(0.75);
  p.c_isq_bias = enc(0.05);
  p.c_isq_g = enc(0.3);
  p.c_log_lin = enc(1.0 / 120.0);
  return p;
}

void erf_coefs(ApproxParams& p) {
  const double two_over_sqrt_pi = 2.0 / std::sqrt(M_PI);
  double fact = 1.0;
  for (int k = 0; k <= p.terms; ++k) {
    if (k > 0) fact *= (double)k;
    const double sgn = (k & 1) ? -1.0 : 1.0;
    p.coef[k] = enc(two_over_sqrt_pi * sgn / (fact * (double)(2 * k + 1)));
  }
}

void log_coefs(ApproxParams& p) {
  for (int k = 1; k <= p.terms; ++k) p.coef[k] = enc(1.0 / (double)k);
}

template <int FN>
int launch_approx(const char* name, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                  uint64_t op_id, const ApproxParams& p, const Cost& cost, void* stream) {
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y, "null pointer");
  int rc;
  {
    KernelTimer timer(name, as_stream(stream));
    approx_kernel<FN><<<grid_for(n, kThreads, 148 * 8), kThreads, 0, as_stream(stream)>>>(
        n, (const u64*)X, (u64*)Y, seed, op_id, p);
    rc = check_launch(name);
  }
  if (rc == MPC_OK) stats_add(cost.rounds, cost.opened, cost.and_gates, cost.words, 0);
  return rc;
}

int check_common(int P, int64_t n) {
  if (P != 2) return fail(MPC_EUNSUPPORTED, "function approximations are implemented for two parties");
  MPC_REQUIRE(n >= 0, "negative length");
  return MPC_OK;
}

#define MPC_APPROX_CHECK(P, n)            \
  do {                                    \
    const int rc_ = check_common(P, n);   \
    if (rc_ != MPC_OK) return rc_;        \
  } while (0)

int check_iters(int exp_iters, int nr_iters) {
  MPC_REQUIRE(exp_iters >= 1 && exp_iters <= MPC_APPROX_MAX_EXP_ITERS, "exp iterations out of range");
  MPC_REQUIRE(nr_iters >= 0 && nr_iters <= MPC_APPROX_MAX_NR_ITERS,
              "Newton-Raphson iterations out of range");
  return MPC_OK;
}

#define MPC_ITERS_CHECK(e, r)              \
  do {                                     \
    const int rc_ = check_iters(e, r);     \
    if (rc_ != MPC_OK) return rc_;         \
  } while (0)

void cost_exp(Cost& c, uint64_t n, int iters) { c.square(n, iters); }
void cost_recip_pos(Cost& c, uint64_t n, int e, int r) {
  cost_exp(c, n, e);
  c.mul(n, 2ull * r);
}
void cost_sigmoid(Cost& c, uint64_t n, int e, int r) {
  c.ltz(n);
  c.mul(n);
  cost_exp(c, n, e);
  c.mul(n, 2ull * r);
  c.mul(n);
}
void cost_inv_sqrt(Cost& c, uint64_t n, int e, int r) {
  cost_exp(c, n, e);
  c.square(n, 4);
  for (int i = 0; i < r; ++i) {
    c.square(n);
    c.mul(n, 2);
  }
}

size_t level_words(int64_t rows, int64_t m) { return 2ull * (size_t)rows * (size_t)((m + 1) / 2); }

// Runs the max tree; returns the [2][rows] maximum (in `ws` or X itself when m == 1).
const u64* run_max_tree(int64_t rows, int64_t m, const u64* X, u64* ws, uint64_t seed,
                        uint64_t& op, Cost& cost, cudaStream_t s, int& rc) {
  const u64* cur = X;
  u64* bufs[2] = {ws, ws + level_words(rows, m)};
  int which = 0;
  rc = MPC_OK;
  while (m > 1) {
    const i64 npairs = m / 2;
    const i64 work = rows * npairs > rows ? rows * npairs : rows;
    u64* out = bufs[which];
    max_level_kernel<<<grid_for(work, kThreads, 148 * 8), kThreads, 0, s>>>(rows, m, cur, out,
                                                                           seed, op);
    rc = check_launch("max_level");
    if (rc != MPC_OK) return nullptr;
    cost.relu((uint64_t)(rows * npairs));
    op += 10;
    cur = out;
    which ^= 1;
    m -= npairs;
  }
  return cur;
}

}  // namespace
}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_exp(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(iters, 0);
  Cost c;
  cost_exp(c, (uint64_t)n, iters);
  return launch_approx<kExp>("approx_exp", n, X, Y, seed, op_id, make_params(iters, 0, 0, 0), c,
                             stream);
}

int mpc_reciprocal(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                   uint64_t op_id, int all_positive, int exp_iters, int nr_iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  const ApproxParams p = make_params(exp_iters, nr_iters, 0, 0);
  Cost c;
  if (all_positive) {
    cost_recip_pos(c, (uint64_t)n, exp_iters, nr_iters);
    return launch_approx<kRecipPos>("approx_reciprocal", n, X, Y, seed, op_id, p, c, stream);
  }
  c.ltz((uint64_t)n);
  c.mul((uint64_t)n);
  cost_recip_pos(c, (uint64_t)n, exp_iters, nr_iters);
  c.mul((uint64_t)n);
  return launch_approx<kRecip>("approx_reciprocal", n, X, Y, seed, op_id, p, c, stream);
}

int mpc_sigmoid(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
                int exp_iters, int nr_iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  Cost c;
  cost_sigmoid(c, (uint64_t)n, exp_iters, nr_iters);
  return launch_approx<kSigmoid>("approx_sigmoid", n, X, Y, seed, op_id,
                                 make_params(exp_iters, nr_iters, 0, 0), c, stream);
}

int mpc_tanh(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
             int exp_iters, int nr_iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  Cost c;
  cost_sigmoid(c, (uint64_t)n, exp_iters, nr_iters);
  return launch_approx<kTanh>("approx_tanh", n, X, Y, seed, op_id,
                              make_params(exp_iters, nr_iters, 0, 0), c, stream);
}

int mpc_erf(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int terms, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_REQUIRE(terms >= 0 && terms < kMaxCoef, "erf terms out of range");
  ApproxParams p = make_params(1, 0, terms, 0);
  erf_coefs(p);
  Cost c;
  c.square((uint64_t)n);
  c.mul((uint64_t)n, (uint64_t)terms);
  return launch_approx<kErf>("approx_erf", n, X, Y, seed, op_id, p, c, stream);
}

int mpc_inv_sqrt(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                 uint64_t op_id, int exp_iters, int nr_iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  Cost c;
  cost_inv_sqrt(c, (uint64_t)n, exp_iters, nr_iters);
  return launch_approx<kInvSqrt>("approx_inv_sqrt", n, X, Y, seed, op_id,
                                 make_params(exp_iters, nr_iters, 0, 0), c, stream);
}

int mpc_sqrt(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
             int exp_iters, int nr_iters, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  Cost c;
  cost_inv_sqrt(c, (uint64_t)n, exp_iters, nr_iters);
  c.mul((uint64_t)n);
  return launch_approx<kSqrt>("approx_sqrt", n, X, Y, seed, op_id,
                              make_params(exp_iters, nr_iters, 0, 0), c, stream);
}

int mpc_log(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int exp_iters, int iters, int order, void* stream) {
  MPC_APPROX_CHECK(P, n);
  MPC_ITERS_CHECK(exp_iters, 0);
  MPC_REQUIRE(iters >= 0 && iters <= MPC_APPROX_MAX_NR_ITERS, "Householder iterations out of range");
  MPC_REQUIRE(order >= 1 && order < kMaxCoef, "Householder order out of range");
  ApproxParams p = make_params(exp_iters, 0, order, iters);
  log_coefs(p);
  Cost c;
  cost_exp(c, (uint64_t)n, exp_iters * (iters + 1));
  c.mul((uint64_t)n, (uint64_t)order * iters);
  return launch_approx<kLog>("approx_log", n, X, Y, seed, op_id, p, c, stream);
}

size_t mpc_max_workspace_size(int P, int64_t rows, int64_t m) {
  if (P != 2 || rows < 0 || m < 1) return 0;
  return 2 * level_words(rows, m) * sizeof(uint64_t);
}

int mpc_max_lastdim(int P, int64_t rows, int64_t m, const uint64_t* X, uint64_t* out,
                    void* workspace, size_t ws_bytes, uint64_t seed, uint64_t op_id,
                    void* stream) {
  MPC_APPROX_CHECK(P, rows);
  MPC_REQUIRE(m >= 1, "empty axis");
  if (rows == 0) return MPC_OK;
  MPC_REQUIRE(X && out, "null pointer");
  MPC_REQUIRE(m == 1 || (workspace && ws_bytes >= mpc_max_workspace_size(P, rows, m)),
              "workspace too small");
  cudaStream_t s = as_stream(stream);
  Cost cost;
  uint64_t op = op_id;
  int rc;
  const u64* mx;
  {
    KernelTimer timer("max_lastdim", s);
    mx = run_max_tree(rows, m, (const u64*)X, (u64*)workspace, seed, op, cost, s, rc);
    if (rc != MPC_OK) return rc;
    if (cudaMemcpyAsync(out, mx, 2ull * rows * sizeof(u64), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return fail(MPC_ECUDA, "copy of the maximum failed");
  }
  stats_add(cost.rounds, cost.opened, cost.and_gates, cost.words, 0);
  return MPC_OK;
}

size_t mpc_softmax_workspace_size(int P, int64_t rows, int64_t m) {
  if (P != 2 || rows < 0 || m < 1) return 0;
  return (2 * level_words(rows, m) + 4ull * (size_t)rows) * sizeof(uint64_t);
}

int mpc_softmax(int P, int64_t rows, int64_t m, const uint64_t* X, uint64_t* Y, void* workspace,
                size_t ws_bytes, uint64_t seed, uint64_t op_id, int exp_iters, int nr_iters,
                void* stream) {
  MPC_APPROX_CHECK(P, rows);
  MPC_ITERS_CHECK(exp_iters, nr_iters);
  MPC_REQUIRE(m >= 1, "empty axis");
  if (rows == 0) return MPC_OK;
  MPC_REQUIRE(X && Y && workspace, "null pointer");
  MPC_REQUIRE(ws_bytes >= mpc_softmax_workspace_size(P, rows, m), "workspace too small");
  MPC_REQUIRE(X != Y, "softmax does not run in place");
  cudaStream_t s = as_stream(stream);
  u64* ws = (u64*)workspace;
  u64* S = ws + 2 * level_words(rows, m);
  u64* R = S + 2 * rows;
  const i64 n = rows * m;
  Cost cost;
  uint64_t op = op_id;
  int rc;
  {
    KernelTimer timer("softmax", s);
    const u64* mx = run_max_tree(rows, m, (const u64*)X, ws, seed, op, cost, s, rc);
    if (rc != MPC_OK) return rc;
    if (cudaMemsetAsync(S, 0, 2ull * rows * sizeof(u64), s) != cudaSuccess)
      return fail(MPC_ECUDA, "memset failed");
    softmax_exp_kernel<<<grid_for(n, kThreads, 148 * 8), kThreads, 0, s>>>(
        rows, m, (const u64*)X, mx, (u64*)Y, S, seed, op, exp_iters);
    if ((rc = check_launch("softmax_exp")) != MPC_OK) return rc;
    cost_exp(cost, (uint64_t)n, exp_iters);
    op += 10ull * exp_iters;
    approx_kernel<kRecipPos><<<grid_for(rows, kThreads, 148 * 8), kThreads, 0, s>>>(
        rows, S, R, seed, op, make_params(exp_iters, nr_iters, 0, 0));
    if ((rc = check_launch("softmax_reciprocal")) != MPC_OK) return rc;
    cost_recip_pos(cost, (uint64_t)rows, exp_iters, nr_iters);
    op += 10ull * exp_iters + 20ull * nr_iters;
    row_scale_kernel<<<grid_for(n, kThreads, 148 * 8), kThreads, 0, s>>>(rows, m, (const u64*)Y,
                                                                         R, (u64*)Y, seed, op);
    if ((rc = check_launch("softmax_scale")) != MPC_OK) return rc;
    cost.mul((uint64_t)n);
  }
  stats_add(cost.rounds, cost.opened, cost.and_gates, cost.words, 0);
  return MPC_OK;
}

}  // extern "C"
