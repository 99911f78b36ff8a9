// Beaver matmul / conv and their dealer triples (App. D.1.1: the Beaver
// identity holds for any bilinear f).  Opening pre-passes, im2col and dealer
// fills live here; the ring GEMM itself is one of the two engines.
//
// Regrouping used for every party p (bit-identical mod 2^64):
//   Z_p = C_p + E B_p + A_p F + [p = 0] E F = C_p + E (B_p + [p = 0] F) + A_p F
// so each party runs one two-pair ring GEMM.  For conv, f(x, w) = W_mat *
// im2col(x), which gives Z_p = C_p + (B_p + [p=0] F)_mat im2col(E) + F_mat im2col(A_p).
#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int kThreads = 256;

// out[i] = sum_p (X_p[i] - A_p[i]) (opening); if G: G[i] = B0[i] + out[i].
template <int P>
__global__ void __launch_bounds__(kThreads) open_kernel(i64 n, const u64* __restrict__ X,
                                                        const u64* __restrict__ A,
                                                        u64* __restrict__ out,
                                                        const u64* __restrict__ B0,
                                                        u64* __restrict__ G) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    u64 e = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) e += X[(i64)p * n + i] - A[(i64)p * n + i];
    out[i] = e;
    if (G) G[i] = B0[i] + e;
  }
}

template <int P>
void launch_open(i64 n, const u64* X, const u64* A, u64* out, const u64* B0, u64* G,
                 cudaStream_t s) {
  open_kernel<P><<<grid_for(n, kThreads), kThreads, 0, s>>>(n, X, A, out, B0, G);
}

// Dealer fill: Out[p] = stream(role, p) for all p and, if sum != null,
// sum = sum_p Out[p].  One thread per Philox block.
__global__ void __launch_bounds__(kThreads) fill_sum_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                            unsigned role, u64* __restrict__ Out,
                                                            u64* __restrict__ sum) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    if (P == 2) {  // both blocks independent (instruction-level parallelism), 16-byte stores
      const u64x4 r0 = prg_block(seed, op_id, stream_word2(role, 0, 0), t);
      const u64x4 r1 = prg_block(seed, op_id, stream_word2(role, 0, 1), t);
      store4(Out, i0, n, as_quad(r0));
      store4(Out + n, i0, n, as_quad(r1));
      if (sum) {
        Quad q;
#pragma unroll
        for (int j = 0; j < 4; ++j) q.v[j] = r0.v[j] + r1.v[j];
        store4(sum, i0, n, q);
      }
      continue;
    }
    u64 acc[4] = {0, 0, 0, 0};
    for (int p = 0; p < P; ++p) {
      const u64x4 r = prg_block(seed, op_id, stream_word2(role, 0, p), t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) Out[(i64)p * n + i0 + j] = r.v[j];
        acc[j] += r.v[j];
      }
    }
    if (sum) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j < n) sum[i0 + j] = acc[j];
    }
  }
}

// The two-party dealer fill with one Philox block per lane: lanes 2j and 2j + 1
// of a warp produce parties 0 and 1 of one 4-word group, and the pair's sum
// is formed with one shuffle.  Twice the threads of fill_sum_kernel's P = 2
// path for the same blocks: a fill of a few hundred thousand words otherwise
// runs a few warps per SM, too few to hide the Philox rounds' latency.  The
// loop runs over whole warps so that every lane takes part in the shuffles.
__global__ void __launch_bounds__(kThreads) fill_sum2_kernel(i64 n, u64 seed, u64 op_id,
                                                             unsigned role, u64* __restrict__ Out,
                                                             u64* __restrict__ sum) {
  const i64 nblk = ceil_div(n, 4);
  const int lane = threadIdx.x & 31, p = lane & 1;
  const i64 wstride = (i64)gridDim.x * blockDim.x;
  for (i64 wb = (blockIdx.x * (i64)blockDim.x + threadIdx.x) - lane; wb < 2 * nblk;
       wb += wstride) {
    const i64 t = (wb + lane) >> 1;
    const bool valid = t < nblk;
    const u64x4 r = prg_block(seed, op_id, stream_word2(role, 0, p), valid ? t : 0);
    const i64 i0 = 4 * t;
    if (valid) store4(Out + (i64)p * n, i0, n, as_quad(r));
    if (sum) {
      Quad q;
#pragma unroll
      for (int j = 0; j < 4; ++j) q.v[j] = r.v[j] + __shfl_xor_sync(0xffffffffu, r.v[j], 1);
      if (valid && p == 0) store4(sum, i0, n, q);
    }
  }
}

// Several two-party dealer fills in one launch (the A and B fills of a batch
// of triples): segment q is fill_sum2_kernel's work for (n, op_id, role, Out,
// sum) of that segment; each segment's lanes are rounded up to whole warps so
// that a warp stays in one segment.
constexpr int kMaxFillSegs = 2 * MPC_MAX_TRIPLE_BATCH;
struct FillSegs {
  u64* Out[kMaxFillSegs];
  u64* sum[kMaxFillSegs];
  i64 n[kMaxFillSegs];
  u64 op_id[kMaxFillSegs];
  unsigned role[kMaxFillSegs];
  i64 base[kMaxFillSegs + 1];  // first lane of each segment (multiples of 32), then the total
  int count;
};

__global__ void __launch_bounds__(kThreads) fill_sum2_multi_kernel(const __grid_constant__ FillSegs f,
                                                                   u64 seed) {
  const int lane = threadIdx.x & 31, p = lane & 1;
  const i64 wstride = (i64)gridDim.x * blockDim.x;
  for (i64 wb = (blockIdx.x * (i64)blockDim.x + threadIdx.x) - lane; wb < f.base[f.count];
       wb += wstride) {
    int q = 0;
    while (wb >= f.base[q + 1]) ++q;
    const i64 n = f.n[q], nblk = ceil_div(n, 4);
    const i64 t = (wb - f.base[q] + lane) >> 1;
    const bool valid = t < nblk;
    const u64x4 r = prg_block(seed, f.op_id[q], stream_word2(f.role[q], 0, p), valid ? t : 0);
    const i64 i0 = 4 * t;
    if (valid) store4(f.Out[q] + (i64)p * n, i0, n, as_quad(r));
    if (f.sum[q]) {
      Quad s4;
#pragma unroll
      for (int j = 0; j < 4; ++j) s4.v[j] = r.v[j] + __shfl_xor_sync(0xffffffffu, r.v[j], 1);
      if (valid && p == 0) store4(f.sum[q], i0, n, s4);
    }
  }
}

// Launches the dealer fill (two parties: fill_sum2_kernel).
int launch_fill_sum(int P, i64 n, u64 seed, u64 op_id, unsigned role, u64* Out, u64* sum,
                    cudaStream_t s) {
  if (n <= 0) return MPC_OK;
  if (P == 2)
    fill_sum2_kernel<<<grid_for(2 * ceil_div(n, 4), kThreads), kThreads, 0, s>>>(n, seed, op_id,
                                                                                 role, Out, sum);
  else
    fill_sum_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, s>>>(P, n, seed, op_id,
                                                                             role, Out, sum);
  return check_launch("dealer fill");
}

// The dealer fills of segments q < count (Out[q], sum[q], n[q], op_id[q],
// role[q]): one launch for two parties, one per segment otherwise.
int launch_fill_multi(int P, int count, u64* const* Out, u64* const* sum, const i64* n,
                      const u64* op_id, const unsigned* role, u64 seed, cudaStream_t s) {
  if (P != 2 || count > kMaxFillSegs) {
    for (int q = 0; q < count; ++q)
      if (int rc = launch_fill_sum(P, n[q], seed, op_id[q], role[q], Out[q], sum[q], s)) return rc;
    return MPC_OK;
  }
  FillSegs f;
  memset(&f, 0, sizeof(f));
  f.count = count;
  for (int q = 0; q < count; ++q) {
    f.Out[q] = Out[q];
    f.sum[q] = sum[q];
    f.n[q] = n[q];
    f.op_id[q] = op_id[q];
    f.role[q] = role[q];
    f.base[q + 1] = f.base[q] + ceil_div(2 * ceil_div(n[q], 4), 32) * 32;
  }
  if (f.base[count] == 0) return MPC_OK;
  fill_sum2_multi_kernel<<<grid_for(f.base[count], kThreads), kThreads, 0, s>>>(f, seed);
  return check_launch("dealer fill");
}

// A triple's two fills (A with its sum a over nA words, B with b over nB).
int launch_fill_pair(int P, u64 seed, u64 op_id, u64* A, u64* a, i64 nA, u64* B, u64* b, i64 nB,
                     cudaStream_t s) {
  u64* out[2] = {A, B};
  u64* sum[2] = {a, b};
  const i64 n[2] = {nA, nB};
  const u64 op[2] = {op_id, op_id};
  const unsigned role[2] = {MPC_ROLE_TRIPLE_A, MPC_ROLE_TRIPLE_B};
  return launch_fill_multi(P, 2, out, sum, n, op, role, seed, s);
}


// Dealer correction: C[p] = stream(TRIPLE_C, p) for p < P-1 and C[P-1] =
// c - sum_{p<P-1} C[p].  c is C[P-1] on entry, or, when the product's GEMM was
// split along K (part != null), the sum of its `splits` partial sums
// part[s * pstride + row * N + col] at the GEMM position (row, col) of each
// output index (the NCHW scatter of gemm_out_index when hw_out != 0): the
// reduction kernel is folded in.  blockIdx.y is the job j of a batch of
// products: C = Cs.C[j], op_id = Cs.op_id[j], part + j n.
struct ShareJobs {
  u64* C[MPC_MAX_TRIPLE_BATCH];
  u64 op_id[MPC_MAX_TRIPLE_BATCH];
};

__global__ void __launch_bounds__(kThreads) share_product_kernel(int P, i64 n, u64 seed,
                                                                 const __grid_constant__ ShareJobs
                                                                     Cs,
                                                                 const u64* __restrict__ part0,
                                                                 i64 pstride, int splits, i64 M,
                                                                 i64 N, i64 hw_out) {
  const int job = blockIdx.y;
  u64* __restrict__ C = Cs.C[job];
  const u64 op_id = Cs.op_id[job];
  const u64* __restrict__ part = part0 ? part0 + (i64)job * n : nullptr;
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    u64 acc[4] = {0, 0, 0, 0};
    for (int p = 0; p < P - 1; ++p) {
      const u64x4 r = prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_C, 0, p), t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) C[(i64)p * n + i0 + j] = r.v[j];
        acc[j] += r.v[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const i64 i = i0 + j;
      if (i >= n) continue;
      u64 c;
      if (part) {
        i64 row, col;
        if (hw_out) {  // i = (b M + row) hw + pos, col = b hw + pos
          const i64 q = i / hw_out, pos = i - q * hw_out;
          const i64 b = q / M;
          row = q - b * M;
          col = b * hw_out + pos;
        } else {
          row = i / N;
          col = i - row * N;
        }
        c = 0;
        for (int sp = 0; sp < splits; ++sp) c += part[(i64)sp * pstride + row * N + col];
      } else {
        c = C[(i64)(P - 1) * n + i];
      }
      C[(i64)(P - 1) * n + i] = c - acc[j];
    }
  }
}

// The dealer's products c_j of the jobs j < used.njobs of a GEMM set (as
// launched, splits deferred: partial sums [splits][njobs][M][N]) shared out as
// C[j] with op ids op_id[j], in one launch.
int share_products(int P, const GemmArgs& used, u64 seed, const u64* op_id, u64* const* C,
                   cudaStream_t s) {
  const i64 n = used.M * used.N;
  const bool split = used.splits > 1;
  ShareJobs Cs;
  memset(&Cs, 0, sizeof(Cs));
  for (int j = 0; j < used.njobs; ++j) {
    Cs.C[j] = C[j];
    Cs.op_id[j] = op_id[j];
  }
  const dim3 grid(grid_for(ceil_div(n, 4), kThreads, 148 * 32 / used.njobs), used.njobs);
  share_product_kernel<<<grid, kThreads, 0, s>>>(P, n, seed, Cs, split ? used.partial : nullptr,
                                                 (i64)used.njobs * n, split ? used.splits : 1,
                                                 used.M, used.N, used.hw_out);
  return check_launch("share product");
}

// The same for a one-job GEMM set.
int share_product(int P, const GemmArgs& used, u64 seed, u64 op_id, u64* C, cudaStream_t s) {
  return share_products(P, used, seed, &op_id, &C, s);
}

// im2col over the ring: col[k][c] with k = (ci * kh + r) * kw + s and
// c = (b * ho + oh) * wo + ow, value = sum_{q < nsrc} (src_q - sub_q) at data
// position (b, ci, oh * sh + r - ph, ow * sw + s - pw), 0 in the padding.
// sub may be null (no subtraction).  src_q = src + q * src_stride.
struct Im2colSrc {
  const u64* src;
  const u64* sub;
  i64 stride;  // elements between consecutive parties
  int nsrc;
};

__global__ void __launch_bounds__(kThreads) im2col_kernel(mpc_conv_desc d, i64 ho, i64 wo,
                                                          Im2colSrc in, u64* __restrict__ col) {
  const i64 ncol = d.batch * ho * wo;
  const i64 K = d.c_in * d.kh * d.kw;
  const i64 total = K * ncol;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const i64 k = i / ncol, c = i % ncol;
    const i64 s = k % d.kw, r = (k / d.kw) % d.kh, ci = k / (d.kw * d.kh);
    const i64 ow = c % wo, oh = (c / wo) % ho, b = c / (wo * ho);
    const i64 y = oh * d.stride_h + r - d.pad_h, x = ow * d.stride_w + s - d.pad_w;
    u64 v = 0;
    if (y >= 0 && y < d.h && x >= 0 && x < d.w) {
      const i64 off = ((b * d.c_in + ci) * d.h + y) * d.w + x;
      for (int q = 0; q < in.nsrc; ++q) {
        v += in.src[q * in.stride + off];
        if (in.sub) v -= in.sub[q * in.stride + off];
      }
    }
    col[i] = v;
  }
}

int launch_im2col(const mpc_conv_desc& d, i64 ho, i64 wo, const Im2colSrc& in, u64* col,
                  cudaStream_t s) {
  const i64 total = d.c_in * d.kh * d.kw * d.batch * ho * wo;
  if (total == 0) return MPC_OK;
  im2col_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(d, ho, wo, in, col);
  return check_launch("im2col");
}

int validate_conv(const mpc_conv_desc* d, i64* ho, i64* wo) {
  MPC_REQUIRE(d != nullptr, "null conv descriptor");
  MPC_REQUIRE(d->batch >= 1 && d->c_in >= 1 && d->h >= 1 && d->w >= 1 && d->c_out >= 1 &&
                  d->kh >= 1 && d->kw >= 1,
              "conv sizes must be positive");
  MPC_REQUIRE(d->stride_h >= 1 && d->stride_w >= 1, "conv strides must be >= 1");
  MPC_REQUIRE(d->pad_h >= 0 && d->pad_w >= 0, "conv padding must be >= 0");
  const i64 lim = 1ll << 31;  // each field in int32 range, so the sums below cannot wrap
  if (d->batch >= lim || d->c_in >= lim || d->h >= lim || d->w >= lim || d->c_out >= lim ||
      d->kh >= lim || d->kw >= lim || d->stride_h >= lim || d->stride_w >= lim ||
      d->pad_h >= lim || d->pad_w >= lim)
    return fail(MPC_EUNSUPPORTED, "conv descriptor field at or above 2^31");
  MPC_REQUIRE(d->h + 2 * d->pad_h >= d->kh && d->w + 2 * d->pad_w >= d->kw,
              "kernel larger than the padded input");
  *ho = (d->h + 2 * d->pad_h - d->kh) / d->stride_h + 1;
  *wo = (d->w + 2 * d->pad_w - d->kw) / d->stride_w + 1;
  // GEMM view M = c_out, K = c_in kh kw, N = batch ho wo and the data size, all
  // bounded before any workspace formula multiplies them.
  if (!mul_fits(d->c_in, d->kh) || !mul_fits(d->c_in * d->kh, d->kw) ||
      !mul_fits(d->batch, *ho) || !mul_fits(d->batch * *ho, *wo) ||
      !mul_fits(d->batch, d->c_in) || !mul_fits(d->batch * d->c_in, d->h) ||
      !mul_fits(d->batch * d->c_in * d->h, d->w) ||
      !gemm_shape_fits(d->c_out, d->batch * *ho * *wo, d->c_in * d->kh * d->kw))
    return fail(MPC_EUNSUPPORTED, "conv shape too large (a size product exceeds 2^52 words)");
  return MPC_OK;
}

// AUTO: the tensor-core limb engine from about a million ring MACs up (it is
// 3-4x faster than the plain engine from 1024^3 on); the plain engine below,
// where launch and plane pre-pass costs dominate.
int resolve_algo(int algo, i64 M, i64 N, i64 K) {
  if (algo != MPC_ALGO_AUTO) return algo;
  return (limb_supported(M, N, K) && (double)M * N * K >= 1048576.0) ? MPC_ALGO_LIMB
                                                                     : MPC_ALGO_PLAIN;
}

inline size_t words(i64 n) { return (size_t)n * sizeof(u64); }
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int engine_splits(int algo, i64 M, i64 N, i64 K, int npairs, int njobs, bool batch) {
  return algo == MPC_ALGO_LIMB ? limb_splits(M, N, K, npairs, njobs, batch)
                               : plain_splits(M, N, K, npairs, njobs);
}

// Engine workspace: split-K partial sums, then (limb) the digit planes.
size_t engine_ws(int algo, i64 M, i64 N, i64 K, int npairs, int njobs, bool batch) {
  const int sp = engine_splits(algo, M, N, K, npairs, njobs, batch);
  size_t b = align256(partial_bytes(sp, njobs, M, N));
  if (algo == MPC_ALGO_LIMB) b += limb_workspace_bytes(M, N, K, npairs, njobs);
  return b;
}

int run_gemm(GemmArgs g, int algo, void* ws, size_t ws_bytes, cudaStream_t s, GemmArgs* used) {
  if (g.M <= 0 || g.N <= 0 || g.njobs <= 0) return MPC_OK;
  const int npairs = g.jobs[0].A2 ? 2 : 1;
  g.splits = engine_splits(algo, g.M, g.N, g.K, npairs, g.njobs, g.gather_per_job != 0);
  if (g.max_splits > 0 && g.splits > g.max_splits) g.splits = g.max_splits;
  const size_t pb = align256(partial_bytes(g.splits, g.njobs, g.M, g.N));
  if (ws_bytes < pb) return fail(MPC_ENOMEM, "engine workspace too small for split-K partials");
  g.partial = g.splits > 1 ? static_cast<u64*>(ws) : nullptr;
  if (used) *used = g;
  void* rest = static_cast<char*>(ws) + pb;
  if (algo == MPC_ALGO_LIMB) return launch_gemm_limb(g, rest, ws_bytes - pb, s);
  return launch_gemm_plain(g, s);
}

namespace {

// Workspace carving (each region 256-byte aligned).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* p) : base(static_cast<char*>(p)) {}
  u64* take(i64 nwords) {
    u64* p = reinterpret_cast<u64*>(base + off);
    off += align256(words(nwords));
    return p;
  }
  void* rest() { return base + off; }
};

size_t matmul_ws(int P, i64 M, i64 N, i64 K, int algo) {
  (void)P;
  return align256(words(M * K)) + 2 * align256(words(K * N)) + engine_ws(algo, M, N, K, 2, P);
}

// The limb engine gathers im2col straight into its digit planes, so only the
// plain engine needs the materialised im2col(E) and im2col(A_p).
size_t conv_ws(int P, const mpc_conv_desc& d, i64 ho, i64 wo, int algo) {
  const i64 M = d.c_out, K = d.c_in * d.kh * d.kw, N = d.batch * ho * wo;
  const size_t cols = algo == MPC_ALGO_LIMB ? 0 : (size_t)(P + 1) * align256(words(K * N));
  return cols + 2 * align256(words(M * K)) + engine_ws(algo, M, N, K, 2, P);
}

size_t matmul_triple_ws(i64 M, i64 N, i64 K, int algo) {
  return align256(words(M * K)) + align256(words(K * N)) + engine_ws(algo, M, N, K, 1, 1);
}

size_t conv_triple_ws(const mpc_conv_desc& d, i64 ho, i64 wo, int algo) {
  const i64 M = d.c_out, K = d.c_in * d.kh * d.kw, N = d.batch * ho * wo;
  const i64 nx = d.batch * d.c_in * d.h * d.w;
  const size_t cols = algo == MPC_ALGO_LIMB ? 0 : align256(words(K * N));
  return align256(words(nx)) + cols + align256(words(M * K)) + engine_ws(algo, M, N, K, 1, 1);
}

int check_algo(int algo) {
  MPC_REQUIRE(algo == MPC_ALGO_PLAIN || algo == MPC_ALGO_LIMB || algo == MPC_ALGO_AUTO,
              "unknown algo %d", algo);
  return MPC_OK;
}

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" {

size_t mpc_matmul_workspace_size(int P, int64_t M, int64_t N, int64_t K, int algo) {
  if (P < 1 || P > MPC_MAX_PARTIES || !gemm_shape_fits(M, N, K)) return 0;
  return matmul_ws(P, M, N, K, resolve_algo(algo, M, N, K));
}

int mpc_beaver_matmul(int P, int64_t M, int64_t N, int64_t K, const uint64_t* X,
                      const uint64_t* Y, const uint64_t* A, const uint64_t* B, const uint64_t* C,
                      uint64_t* Z, int algo, int trunc_bits, void* ws, size_t ws_bytes,
                      void* stream) {
  MPC_CHECK_PARTIES(P);
  if (int rc = check_algo(algo)) return rc;
  MPC_REQUIRE(M >= 0 && N >= 0 && K >= 0, "negative dimension");
  if (!gemm_shape_fits(M, N, K))
    return fail(MPC_EUNSUPPORTED, "shape too large: M*K, K*N or M*N exceeds 2^52 words");
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  if (M == 0 || N == 0) return MPC_OK;
  // With K = 0 the operands and a, b are empty (never read) and may be NULL.
  MPC_REQUIRE(C && Z && (K == 0 || (X && Y && A && B)), "null pointer");
  algo = resolve_algo(algo, M, N, K);
  if (algo == MPC_ALGO_LIMB && !limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support M=%lld N=%lld K=%lld",
                (long long)M, (long long)N, (long long)K);
  const size_t need = matmul_ws(P, M, N, K, algo);
  MPC_REQUIRE(ws != nullptr || need == 0, "null workspace");
  if (ws_bytes < need)
    return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  u64* E = cv.take(M * K);
  u64* F = cv.take(K * N);
  u64* G = cv.take(K * N);
  if (K > 0) {
    MPC_DISPATCH_P(P, launch_open, M * K, (const u64*)X, (const u64*)A, E, nullptr, nullptr, s);
    if (int rc = check_launch("open E")) return rc;
    MPC_DISPATCH_P(P, launch_open, K * N, (const u64*)Y, (const u64*)B, F, (const u64*)B, G, s);
    if (int rc = check_launch("open F")) return rc;
  }
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.hw_out = 0;
  g.trunc_bits = trunc_bits;
  g.njobs = P;
  for (int p = 0; p < P; ++p) {
    g.jobs[p].A1 = E;
    g.jobs[p].B1 = p == 0 ? G : (const u64*)B + (i64)p * K * N;
    g.jobs[p].A2 = (const u64*)A + (i64)p * M * K;
    g.jobs[p].B2 = F;
    g.jobs[p].C = (const u64*)C + (i64)p * M * N;
    g.jobs[p].Z = (u64*)Z + (i64)p * M * N;
  }
  int rc = run_gemm(g, algo, cv.rest(), ws_bytes - cv.off, s);
  if (rc == MPC_OK)
    stats_add(1, 8ull * (uint64_t)(M * K + K * N), 0, (uint64_t)P * (M * K + K * N + M * N),
              (uint64_t)P * 2ull * M * N * K);
  return rc;
}

size_t mpc_conv2d_workspace_size(int P, const mpc_conv_desc* d, int algo) {
  i64 ho, wo;
  if (P < 1 || P > MPC_MAX_PARTIES || validate_conv(d, &ho, &wo) != MPC_OK) return 0;
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  return conv_ws(P, *d, ho, wo, resolve_algo(algo, M, N, K));
}

}  // extern "C"

namespace mpc {
namespace {

// The Beaver convolution; with `deferred`, a split-K job set leaves its partial
// sums for the caller (the job set as launched is copied there).
// prep (limb engine only): the planes limb_conv_prepare cut from W and B ahead
// of the call; W and B are then not read.
int beaver_conv2d_impl(int P, const mpc_conv_desc* d, const uint64_t* X, const uint64_t* W,
                       const uint64_t* A, const uint64_t* B, const uint64_t* C, uint64_t* Z,
                       int algo, int trunc_bits, void* ws, size_t ws_bytes, void* stream,
                       GemmArgs* deferred, const void* prep = nullptr) {
  MPC_CHECK_PARTIES(P);
  if (int rc = check_algo(algo)) return rc;
  i64 ho, wo;
  if (int rc = validate_conv(d, &ho, &wo)) return rc;
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  MPC_REQUIRE(X && A && C && Z && (prep || (W && B)), "null pointer");
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  const i64 nx = d->batch * d->c_in * d->h * d->w;
  algo = prep ? MPC_ALGO_LIMB : resolve_algo(algo, M, N, K);
  if (algo == MPC_ALGO_LIMB && !limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this conv shape");
  const size_t need = conv_ws(P, *d, ho, wo, algo);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  const bool gather = algo == MPC_ALGO_LIMB;
  u64* Ecol = nullptr;
  u64* Acol[MPC_MAX_PARTIES] = {nullptr};
  if (!gather) {
    Ecol = cv.take(K * N);
    for (int p = 0; p < P; ++p) Acol[p] = cv.take(K * N);
  }
  u64* F = cv.take(M * K);
  u64* G = cv.take(M * K);
  ConvGather cg{};
  if (gather) {
    // The limb engine reads E = sum_p (X_p - A_p) and A_p at their data positions.
    cg.d = *d;
    cg.ho = ho;
    cg.wo = wo;
    cg.src1 = (const u64*)X;
    cg.sub1 = (const u64*)A;
    cg.stride1 = nx;
    cg.n1 = P;
    for (int p = 0; p < P; ++p) cg.src2[p] = (const u64*)A + p * nx;
  } else {
    // E = sum_p (X_p - A_p) gathered straight into im2col layout.
    if (int rc = launch_im2col(*d, ho, wo, Im2colSrc{(const u64*)X, (const u64*)A, nx, P}, Ecol,
                               s))
      return rc;
    for (int p = 0; p < P; ++p)
      if (int rc = launch_im2col(*d, ho, wo, Im2colSrc{(const u64*)A + p * nx, nullptr, nx, 1},
                                 Acol[p], s))
        return rc;
  }
  if (!prep) {
    MPC_DISPATCH_P(P, launch_open, M * K, (const u64*)W, (const u64*)B, F, (const u64*)B, G, s);
    if (int rc = check_launch("open F")) return rc;
  }
  GemmArgs g{};
  g.prep = prep;
  g.M = M;
  g.N = N;
  g.K = K;
  g.hw_out = ho * wo;
  g.trunc_bits = trunc_bits;
  g.njobs = P;
  g.gather = gather ? &cg : nullptr;
  g.defer_reduce = deferred != nullptr;
  for (int p = 0; p < P; ++p) {
    g.jobs[p].A1 = p == 0 ? G : (prep ? nullptr : (const u64*)B + (i64)p * M * K);
    g.jobs[p].B1 = Ecol;
    g.jobs[p].A2 = F;
    g.jobs[p].B2 = Acol[p];
    g.jobs[p].C = (const u64*)C + (i64)p * M * N;
    g.jobs[p].Z = (u64*)Z + (i64)p * M * N;
  }
  int rc = run_gemm(g, algo, cv.rest(), ws_bytes - cv.off, s, deferred);
  // With prepared planes F was opened (and counted) by the prepare call.
  if (rc == MPC_OK)
    stats_add(1, 8ull * (uint64_t)(nx + (prep ? 0 : M * K)), 0,
              (uint64_t)P * (nx + M * K + M * N), (uint64_t)P * 2ull * M * N * K);
  return rc;
}

}  // namespace
}  // namespace mpc

extern "C" {

int mpc_beaver_conv2d(int P, const mpc_conv_desc* d, const uint64_t* X, const uint64_t* W,
                      const uint64_t* A, const uint64_t* B, const uint64_t* C, uint64_t* Z,
                      int algo, int trunc_bits, void* ws, size_t ws_bytes, void* stream) {
  return beaver_conv2d_impl(P, d, X, W, A, B, C, Z, algo, trunc_bits, ws, ws_bytes, stream,
                            nullptr);
}

int mpc_beaver_conv2d_relu(int P, const mpc_conv_desc* d, const uint64_t* X, const uint64_t* W,
                           const uint64_t* A, const uint64_t* B, const uint64_t* C, uint64_t* Y,
                           int algo, int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                           size_t ws_bytes, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "convolution + fused ReLU supports P = 2 (got %d)", P);
  GemmArgs used{};
  used.njobs = 0;
  if (int rc = beaver_conv2d_impl(P, d, X, W, A, B, C, Y, algo, trunc_bits, ws, ws_bytes, stream,
                                  &used))
    return rc;
  if (used.njobs != 2) return fail(MPC_EINVAL, "empty convolution");
  return launch_relu_of_gemm(used, (u64*)Y, seed, relu_op, as_stream(stream));
}

int mpc_beaver_conv2d_relu_add(int P, const mpc_conv_desc* d, const uint64_t* X,
                               const uint64_t* W, const uint64_t* A, const uint64_t* B,
                               const uint64_t* C, const uint64_t* S, uint64_t* Y, int algo,
                               int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                               size_t ws_bytes, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "convolution + residual + fused ReLU supports P = 2 (got %d)", P);
  MPC_REQUIRE(S != nullptr && S != Y, "null residual or residual aliasing the output");
  GemmArgs used{};
  used.njobs = 0;
  if (int rc = beaver_conv2d_impl(P, d, X, W, A, B, C, Y, algo, trunc_bits, ws, ws_bytes, stream,
                                  &used))
    return rc;
  if (used.njobs != 2) return fail(MPC_EINVAL, "empty convolution");
  return launch_relu_of_gemm(used, (u64*)Y, seed, relu_op, as_stream(stream), (const u64*)S);
}

size_t mpc_conv2d_prep_size(int P, const mpc_conv_desc* d) {
  i64 ho, wo;
  if (P < 1 || P > MPC_MAX_PARTIES || validate_conv(d, &ho, &wo) != MPC_OK) return 0;
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  if (!limb_supported(M, N, K)) return 0;
  // the planes, then F and G (the opened weight difference, scratch)
  return limb_conv_prep_bytes(P, M, N, K) + 2 * align256(words(M * K));
}

int mpc_beaver_conv2d_prepare(int P, const mpc_conv_desc* d, const uint64_t* W, const uint64_t* A,
                              const uint64_t* B, void* prep, size_t prep_bytes, void* stream) {
  MPC_CHECK_PARTIES(P);
  i64 ho, wo;
  if (int rc = validate_conv(d, &ho, &wo)) return rc;
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  if (M * N * K == 0) return MPC_OK;
  MPC_REQUIRE(W && A && B && prep, "null pointer");
  if (!limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this conv shape");
  const size_t planes = limb_conv_prep_bytes(P, M, N, K);
  const size_t need = planes + 2 * align256(words(M * K));
  if (prep_bytes < need) return fail(MPC_ENOMEM, "prep buffer %zu bytes, need %zu", prep_bytes, need);
  cudaStream_t s = as_stream(stream);
  u64* F = reinterpret_cast<u64*>(static_cast<char*>(prep) + planes);
  u64* G = F + align256(words(M * K)) / sizeof(u64);
  MPC_DISPATCH_P(P, launch_open, M * K, (const u64*)W, (const u64*)B, F, (const u64*)B, G, s);
  if (int rc = check_launch("open F")) return rc;
  const u64* asrc[MPC_MAX_PARTIES + 1];
  asrc[0] = G;
  for (int p = 1; p < P; ++p) asrc[p] = (const u64*)B + (i64)p * M * K;
  asrc[P] = F;
  ConvGather cg{};
  cg.d = *d;
  cg.ho = ho;
  cg.wo = wo;
  cg.stride1 = d->batch * d->c_in * d->h * d->w;
  cg.n1 = P;
  for (int p = 0; p < P; ++p) cg.src2[p] = (const u64*)A + p * cg.stride1;
  const int rc = limb_conv_prepare(P, cg, M, N, K, asrc, prep, s);
  if (rc == MPC_OK) stats_add(1, 8ull * (uint64_t)(M * K), 0, 0, 0);
  return rc;
}

int mpc_beaver_conv2d_prepared(int P, const mpc_conv_desc* d, const uint64_t* X,
                               const uint64_t* A, const uint64_t* C, const void* prep,
                               size_t prep_bytes, uint64_t* Z, int trunc_bits, void* ws,
                               size_t ws_bytes, void* stream) {
  const size_t need = mpc_conv2d_prep_size(P, d);
  MPC_REQUIRE(prep != nullptr, "null prep buffer");
  if (need == 0) return fail(MPC_EUNSUPPORTED, "no prepared planes for this shape or party count");
  if (prep_bytes < need) return fail(MPC_ENOMEM, "prep buffer %zu bytes, need %zu", prep_bytes, need);
  return beaver_conv2d_impl(P, d, X, nullptr, A, nullptr, C, Z, MPC_ALGO_LIMB, trunc_bits, ws,
                            ws_bytes, stream, nullptr, prep);
}

int mpc_beaver_conv2d_relu_prepared(int P, const mpc_conv_desc* d, const uint64_t* X,
                                    const uint64_t* A, const uint64_t* C, const void* prep,
                                    size_t prep_bytes, uint64_t* Y, int trunc_bits, uint64_t seed,
                                    uint64_t relu_op, void* ws, size_t ws_bytes, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "convolution + fused ReLU supports P = 2 (got %d)", P);
  const size_t need = mpc_conv2d_prep_size(P, d);
  MPC_REQUIRE(prep != nullptr, "null prep buffer");
  if (need == 0) return fail(MPC_EUNSUPPORTED, "no prepared planes for this shape");
  if (prep_bytes < need) return fail(MPC_ENOMEM, "prep buffer %zu bytes, need %zu", prep_bytes, need);
  GemmArgs used{};
  used.njobs = 0;
  if (int rc = beaver_conv2d_impl(P, d, X, nullptr, A, nullptr, C, Y, MPC_ALGO_LIMB, trunc_bits,
                                  ws, ws_bytes, stream, &used, prep))
    return rc;
  if (used.njobs != 2) return fail(MPC_EINVAL, "empty convolution");
  return launch_relu_of_gemm(used, (u64*)Y, seed, relu_op, as_stream(stream));
}

// ---- prepared products: the dealer adds A_p F into C_p --------------------------
namespace {

struct ProdPrep {
  i64 M, N, K, ho, wo, nx;
  size_t planes, cwords;  // bytes of one plane set, of one party's C'
};

int prod_prep_shape(int P, const mpc_conv_desc* d, ProdPrep* q) {
  MPC_CHECK_PARTIES(P);
  i64 ho, wo;
  if (int rc = validate_conv(d, &ho, &wo)) return rc;
  q->M = d->c_out;
  q->K = d->c_in * d->kh * d->kw;
  q->N = d->batch * ho * wo;
  q->ho = ho;
  q->wo = wo;
  q->nx = d->batch * d->c_in * d->h * d->w;
  if (!limb_supported(q->M, q->N, q->K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this conv shape");
  q->planes = limb_planes_a_bytes(q->M, q->K);
  q->cwords = align256(words(q->M * q->N));
  return MPC_OK;
}

// Online half of a convolution on prepared products: E opened and gathered,
// one operand pair per party, C'_p from prep.
int conv_prepared_products_impl(int P, const mpc_conv_desc* d, const uint64_t* X,
                                const uint64_t* A, const void* prep, size_t prep_bytes,
                                uint64_t* Z, int trunc_bits, void* ws, size_t ws_bytes,
                                cudaStream_t s, GemmArgs* deferred) {
  ProdPrep q;
  if (int rc = prod_prep_shape(P, d, &q)) return rc;
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  MPC_REQUIRE(X && A && prep && Z, "null pointer");
  if (prep_bytes < mpc_conv2d_prep_products_size(P, d))
    return fail(MPC_ENOMEM, "prep buffer %zu bytes, too small", prep_bytes);
  const size_t need = engine_ws(MPC_ALGO_LIMB, q.M, q.N, q.K, 1, P);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  const char* cp = static_cast<const char*>(prep) + (size_t)P * q.planes;
  ConvGather cg{};
  cg.d = *d;
  cg.ho = q.ho;
  cg.wo = q.wo;
  cg.src1 = (const u64*)X;
  cg.sub1 = (const u64*)A;
  cg.stride1 = q.nx;
  cg.n1 = P;
  GemmArgs g{};
  g.prep = prep;
  g.prep_pairs = 1;
  g.M = q.M;
  g.N = q.N;
  g.K = q.K;
  g.hw_out = q.ho * q.wo;
  g.trunc_bits = trunc_bits;
  g.njobs = P;
  g.gather = &cg;
  g.defer_reduce = deferred != nullptr;
  for (int p = 0; p < P; ++p) {
    g.jobs[p].C = reinterpret_cast<const u64*>(cp + (size_t)p * q.cwords);
    g.jobs[p].Z = (u64*)Z + (i64)p * q.M * q.N;
  }
  const int rc = run_gemm(g, MPC_ALGO_LIMB, ws, ws_bytes, s, deferred);
  if (rc == MPC_OK)
    stats_add(1, 8ull * (uint64_t)q.nx, 0, (uint64_t)P * (uint64_t)q.nx,
              (uint64_t)P * (uint64_t)(q.M * q.N * q.K));
  return rc;
}

}  // namespace

size_t mpc_conv2d_prep_products_size(int P, const mpc_conv_desc* d) {
  ProdPrep q;
  if (P < 1 || P > MPC_MAX_PARTIES || prod_prep_shape(P, d, &q) != MPC_OK) return 0;
  return (size_t)P * (q.planes + q.cwords);
}

size_t mpc_conv2d_prepare_products_workspace_size(int P, const mpc_conv_desc* d) {
  ProdPrep q;
  if (P < 1 || P > MPC_MAX_PARTIES || prod_prep_shape(P, d, &q) != MPC_OK) return 0;
  return 2 * align256(words(q.M * q.K)) + engine_ws(MPC_ALGO_LIMB, q.M, q.N, q.K, 1, P, true);
}

int mpc_beaver_conv2d_prepare_products(int P, const mpc_conv_desc* d, const uint64_t* W,
                                       const uint64_t* A, const uint64_t* B, const uint64_t* C,
                                       void* prep, size_t prep_bytes, void* ws, size_t ws_bytes,
                                       void* stream) {
  ProdPrep q;
  if (int rc = prod_prep_shape(P, d, &q)) return rc;
  MPC_REQUIRE(W && A && B && C && prep, "null pointer");
  if (prep_bytes < (size_t)P * (q.planes + q.cwords))
    return fail(MPC_ENOMEM, "prep buffer %zu bytes, need %zu", prep_bytes,
                (size_t)P * (q.planes + q.cwords));
  const size_t need = mpc_conv2d_prepare_products_workspace_size(P, d);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  u64* F = cv.take(q.M * q.K);
  u64* G = cv.take(q.M * q.K);
  // F = sum_p (W_p - B_p) opened, G = B_0 + F
  MPC_DISPATCH_P(P, launch_open, q.M * q.K, (const u64*)W, (const u64*)B, F, (const u64*)B, G, s);
  if (int rc = check_launch("open F")) return rc;
  // C'_p = C_p + A_p F: one one-pair job per party, F times its own im2col(A_p)
  char* cp = static_cast<char*>(prep) + (size_t)P * q.planes;
  ConvGather cg[MPC_MAX_PARTIES] = {};
  GemmArgs g{};
  g.M = q.M;
  g.N = q.N;
  g.K = q.K;
  g.hw_out = q.ho * q.wo;
  g.njobs = P;
  g.gather = cg;
  g.gather_per_job = 1;
  for (int p = 0; p < P; ++p) {
    cg[p].d = *d;
    cg[p].ho = q.ho;
    cg[p].wo = q.wo;
    cg[p].src2[0] = (const u64*)A + (i64)p * q.nx;
    g.jobs[p] = GemmJob{F, nullptr, nullptr, nullptr, (const u64*)C + (i64)p * q.M * q.N,
                        reinterpret_cast<u64*>(cp + (size_t)p * q.cwords)};
  }
  if (int rc = run_gemm(g, MPC_ALGO_LIMB, cv.rest(), ws_bytes - cv.off, s, nullptr)) return rc;
  // digit planes of the first-pair weights G, B_1 .. B_{P-1}
  const u64* asrc[MPC_MAX_PARTIES];
  asrc[0] = G;
  for (int p = 1; p < P; ++p) asrc[p] = (const u64*)B + (i64)p * q.M * q.K;
  if (int rc = limb_cut_planes_a(P, asrc, q.M, q.K, prep, s)) return rc;
  stats_add(1, 8ull * (uint64_t)(q.M * q.K), 0, 0, (uint64_t)P * (uint64_t)(q.M * q.N * q.K));
  return MPC_OK;
}

int mpc_beaver_conv2d_prepared_products(int P, const mpc_conv_desc* d, const uint64_t* X,
                                        const uint64_t* A, const void* prep, size_t prep_bytes,
                                        uint64_t* Z, int trunc_bits, void* ws, size_t ws_bytes,
                                        void* stream) {
  return conv_prepared_products_impl(P, d, X, A, prep, prep_bytes, Z, trunc_bits, ws, ws_bytes,
                                     as_stream(stream), nullptr);
}

int mpc_beaver_conv2d_relu_prepared_products(int P, const mpc_conv_desc* d, const uint64_t* X,
                                             const uint64_t* A, const void* prep,
                                             size_t prep_bytes, uint64_t* Y, int trunc_bits,
                                             uint64_t seed, uint64_t relu_op, void* ws,
                                             size_t ws_bytes, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "convolution + fused ReLU supports P = 2 (got %d)", P);
  GemmArgs used{};
  used.njobs = 0;
  if (int rc = conv_prepared_products_impl(P, d, X, A, prep, prep_bytes, Y, trunc_bits, ws,
                                           ws_bytes, as_stream(stream), &used))
    return rc;
  if (used.njobs != 2) return fail(MPC_EINVAL, "empty convolution");
  return launch_relu_of_gemm(used, (u64*)Y, seed, relu_op, as_stream(stream));
}

int mpc_beaver_conv2d_relu_prepared_add(int P, const mpc_conv_desc* d, const uint64_t* X,
                                        const uint64_t* A, const uint64_t* C, const void* prep,
                                        size_t prep_bytes, const uint64_t* S, uint64_t* Y,
                                        int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                                        size_t ws_bytes, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "convolution + residual + fused ReLU supports P = 2 (got %d)", P);
  MPC_REQUIRE(S != nullptr && S != Y, "null residual or residual aliasing the output");
  const size_t need = mpc_conv2d_prep_size(P, d);
  MPC_REQUIRE(prep != nullptr, "null prep buffer");
  if (need == 0) return fail(MPC_EUNSUPPORTED, "no prepared planes for this shape");
  if (prep_bytes < need) return fail(MPC_ENOMEM, "prep buffer %zu bytes, need %zu", prep_bytes, need);
  GemmArgs used{};
  used.njobs = 0;
  if (int rc = beaver_conv2d_impl(P, d, X, nullptr, A, nullptr, C, Y, MPC_ALGO_LIMB, trunc_bits,
                                  ws, ws_bytes, stream, &used, prep))
    return rc;
  if (used.njobs != 2) return fail(MPC_EINVAL, "empty convolution");
  return launch_relu_of_gemm(used, (u64*)Y, seed, relu_op, as_stream(stream), (const u64*)S);
}

size_t mpc_ring_gemm_workspace_size(int64_t M, int64_t N, int64_t K, int algo) {
  if (!gemm_shape_fits(M, N, K)) return 0;
  return engine_ws(resolve_algo(algo, M, N, K), M, N, K, 1, 1);
}

int mpc_ring_gemm(int64_t M, int64_t N, int64_t K, const uint64_t* A, const uint64_t* B,
                  const uint64_t* C, uint64_t* Z, int algo, void* ws, size_t ws_bytes,
                  void* stream) {
  if (int rc = check_algo(algo)) return rc;
  MPC_REQUIRE(M >= 0 && N >= 0 && K >= 0, "negative dimension");
  if (!gemm_shape_fits(M, N, K))
    return fail(MPC_EUNSUPPORTED, "shape too large: M*K, K*N or M*N exceeds 2^52 words");
  if (M == 0 || N == 0) return MPC_OK;
  MPC_REQUIRE(A && B && Z, "null pointer");
  algo = resolve_algo(algo, M, N, K);
  if (algo == MPC_ALGO_LIMB && !limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support M=%lld N=%lld K=%lld",
                (long long)M, (long long)N, (long long)K);
  const size_t need = engine_ws(algo, M, N, K, 1, 1);
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.njobs = 1;
  g.jobs[0] = GemmJob{(const u64*)A, (const u64*)B, nullptr, nullptr, (const u64*)C, (u64*)Z};
  int rc = run_gemm(g, algo, ws, ws_bytes, as_stream(stream));
  if (rc == MPC_OK) stats_add(0, 0, 0, 0, 2ull * M * N * K);
  return rc;
}

size_t mpc_matmul_triple_workspace_size(int P, int64_t M, int64_t N, int64_t K, int algo) {
  if (P < 1 || P > MPC_MAX_PARTIES || !gemm_shape_fits(M, N, K)) return 0;
  return matmul_triple_ws(M, N, K, resolve_algo(algo, M, N, K));
}

int mpc_ttp_matmul_triple(int P, int64_t M, int64_t N, int64_t K, uint64_t seed, uint64_t op_id,
                          uint64_t* A, uint64_t* B, uint64_t* C, int algo, void* ws,
                          size_t ws_bytes, void* stream) {
  MPC_CHECK_PARTIES(P);
  if (int rc = check_algo(algo)) return rc;
  MPC_REQUIRE(M >= 0 && N >= 0 && K >= 0, "negative dimension");
  if (!gemm_shape_fits(M, N, K))
    return fail(MPC_EUNSUPPORTED, "shape too large: M*K, K*N or M*N exceeds 2^52 words");
  MPC_REQUIRE(C && ((A && B) || M * K + K * N == 0), "null pointer");
  algo = resolve_algo(algo, M, N, K);
  if (algo == MPC_ALGO_LIMB && !limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this shape");
  const size_t need = matmul_triple_ws(M, N, K, algo);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  u64* a = cv.take(M * K);
  u64* b = cv.take(K * N);
  if (int rc = launch_fill_pair(P, seed, op_id, (u64*)A, a, M * K, (u64*)B, b, K * N, s)) return rc;
  if (M * N == 0) return MPC_OK;
  u64* Clast = (u64*)C + (i64)(P - 1) * M * N;
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.njobs = 1;
  g.jobs[0] = GemmJob{a, b, nullptr, nullptr, nullptr, Clast};
  g.defer_reduce = 1;  // the correction kernel adds the split-K partial sums itself
  GemmArgs used{};
  if (int rc = run_gemm(g, algo, cv.rest(), ws_bytes - cv.off, s, &used)) return rc;
  return share_product(P, used, seed, op_id, (u64*)C, s);
}

size_t mpc_conv2d_triple_workspace_size(int P, const mpc_conv_desc* d, int algo) {
  i64 ho, wo;
  if (P < 1 || P > MPC_MAX_PARTIES || validate_conv(d, &ho, &wo) != MPC_OK) return 0;
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  return conv_triple_ws(*d, ho, wo, resolve_algo(algo, M, N, K));
}

int mpc_ttp_conv2d_triple(int P, const mpc_conv_desc* d, uint64_t seed, uint64_t op_id,
                          uint64_t* A, uint64_t* B, uint64_t* C, int algo, void* ws,
                          size_t ws_bytes, void* stream) {
  MPC_CHECK_PARTIES(P);
  if (int rc = check_algo(algo)) return rc;
  i64 ho, wo;
  if (int rc = validate_conv(d, &ho, &wo)) return rc;
  MPC_REQUIRE(A && B && C, "null pointer");
  const i64 M = d->c_out, K = d->c_in * d->kh * d->kw, N = d->batch * ho * wo;
  const i64 nx = d->batch * d->c_in * d->h * d->w;
  algo = resolve_algo(algo, M, N, K);
  if (algo == MPC_ALGO_LIMB && !limb_supported(M, N, K))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this conv shape");
  const size_t need = conv_triple_ws(*d, ho, wo, algo);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  const bool gather = algo == MPC_ALGO_LIMB;
  u64* a = cv.take(nx);
  u64* acol = gather ? nullptr : cv.take(K * N);
  u64* b = cv.take(M * K);
  if (int rc = launch_fill_pair(P, seed, op_id, (u64*)A, a, nx, (u64*)B, b, M * K, s)) return rc;
  ConvGather cg{};
  if (gather) {
    cg.d = *d;
    cg.ho = ho;
    cg.wo = wo;
    cg.src1 = a;
    cg.n1 = 1;
  } else if (int rc = launch_im2col(*d, ho, wo, Im2colSrc{a, nullptr, 0, 1}, acol, s)) {
    return rc;
  }
  u64* Clast = (u64*)C + (i64)(P - 1) * M * N;
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.hw_out = ho * wo;
  g.njobs = 1;
  g.gather = gather ? &cg : nullptr;
  g.jobs[0] = GemmJob{b, acol, nullptr, nullptr, nullptr, Clast};
  g.defer_reduce = 1;  // the correction kernel adds the split-K partial sums itself
  GemmArgs used{};
  if (int rc = run_gemm(g, algo, cv.rest(), ws_bytes - cv.off, s, &used)) return rc;
  return share_product(P, used, seed, op_id, (u64*)C, s);
}

// A batch of `count` convolution triples with one output shape (c_out, batch,
// ho, wo).  On the limb engine the count products c_j = conv(a_j, b_j) run
// as the jobs of one GEMM launch, each with its own K (one digit-plane launch
// per run of equal descriptors gathers the a_j); on the plain engine the
// triples are dealt one by one.
namespace {

struct TripleBatch {
  i64 M, N, ho, wo, Kmax;
};

int check_triple_batch(int count, const mpc_conv_desc* d, TripleBatch* b) {
  MPC_REQUIRE(d != nullptr, "null descriptor array");
  i64 ho0, wo0;
  if (int rc = validate_conv(&d[0], &ho0, &wo0)) return rc;
  b->M = d[0].c_out;
  b->N = d[0].batch * ho0 * wo0;
  b->ho = ho0;
  b->wo = wo0;
  b->Kmax = 0;
  for (int j = 0; j < count; ++j) {
    i64 ho, wo;
    if (int rc = validate_conv(&d[j], &ho, &wo)) return rc;
    MPC_REQUIRE(d[j].c_out == d[0].c_out && d[j].batch == d[0].batch && ho == ho0 && wo == wo0,
                "triple %d: output shape differs from triple 0's", j);
    b->Kmax = std::max<i64>(b->Kmax, d[j].c_in * d[j].kh * d[j].kw);
  }
  return MPC_OK;
}

}  // namespace

size_t mpc_conv2d_triples_workspace_size(int P, int count, const mpc_conv_desc* d, int algo) {
  TripleBatch tb;
  if (P < 1 || P > MPC_MAX_PARTIES || count < 1 || count > MPC_MAX_TRIPLE_BATCH ||
      check_algo(algo) != MPC_OK || check_triple_batch(count, d, &tb) != MPC_OK)
    return 0;
  algo = resolve_algo(algo, tb.M, tb.N, tb.Kmax);
  if (algo != MPC_ALGO_LIMB || !limb_supported(tb.M, tb.N, tb.Kmax) || count == 1) {
    size_t need = 0;
    for (int j = 0; j < count; ++j) need = std::max(need, conv_triple_ws(d[j], tb.ho, tb.wo, algo));
    return need;
  }
  size_t need = engine_ws(MPC_ALGO_LIMB, tb.M, tb.N, tb.Kmax, 1, count, true);
  for (int j = 0; j < count; ++j)
    need += align256(words(d[j].batch * d[j].c_in * d[j].h * d[j].w)) +
            align256(words(tb.M * d[j].c_in * d[j].kh * d[j].kw));
  return need;
}

int mpc_ttp_conv2d_triples(int P, int count, const mpc_conv_desc* d, uint64_t seed,
                           const uint64_t* op_ids, uint64_t* const* A, uint64_t* const* B,
                           uint64_t* const* C, int algo, void* ws, size_t ws_bytes,
                           void* stream) {
  MPC_CHECK_PARTIES(P);
  if (int rc = check_algo(algo)) return rc;
  MPC_REQUIRE(count >= 1 && count <= MPC_MAX_TRIPLE_BATCH, "count %d outside [1, %d]", count,
              MPC_MAX_TRIPLE_BATCH);
  TripleBatch tb;
  if (int rc = check_triple_batch(count, d, &tb)) return rc;
  MPC_REQUIRE(op_ids && A && B && C, "null pointer");
  for (int j = 0; j < count; ++j) MPC_REQUIRE(A[j] && B[j] && C[j], "null pointer (triple %d)", j);
  const i64 M = tb.M, N = tb.N;
  algo = resolve_algo(algo, M, N, tb.Kmax);
  if (algo != MPC_ALGO_LIMB || count == 1) {
    for (int j = 0; j < count; ++j)
      if (int rc = mpc_ttp_conv2d_triple(P, &d[j], seed, op_ids[j], A[j], B[j], C[j], algo, ws,
                                         ws_bytes, stream))
        return rc;
    return MPC_OK;
  }
  if (!limb_supported(M, N, tb.Kmax))
    return fail(MPC_EUNSUPPORTED, "limb engine does not support this conv shape");
  const size_t need = mpc_conv2d_triples_workspace_size(P, count, d, algo);
  MPC_REQUIRE(ws != nullptr, "null workspace");
  if (ws_bytes < need) return fail(MPC_ENOMEM, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  Carve cv(ws);
  ConvGather cg[MPC_MAX_TRIPLE_BATCH] = {};
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = tb.Kmax;
  g.hw_out = tb.ho * tb.wo;
  g.njobs = count;
  g.gather = cg;
  g.gather_per_job = 1;
  g.defer_reduce = 1;  // the correction kernels add the split-K partial sums themselves
  g.max_splits = 64;
  // The fills, one launch each: a single launch for all of them made the dealer
  // alone 7 % faster but the overlapped speech step 1 % slower (one wide
  // launch takes every SM from the online phase at once; small ones fit in
  // its gaps).
  u64* fout[2 * MPC_MAX_TRIPLE_BATCH];
  u64* fsum[2 * MPC_MAX_TRIPLE_BATCH];
  i64 fn[2 * MPC_MAX_TRIPLE_BATCH];
  u64 fop[2 * MPC_MAX_TRIPLE_BATCH];
  unsigned frole[2 * MPC_MAX_TRIPLE_BATCH];
  for (int j = 0; j < count; ++j) {
    const i64 nx = d[j].batch * d[j].c_in * d[j].h * d[j].w;
    const i64 K = d[j].c_in * d[j].kh * d[j].kw;
    u64* a = cv.take(nx);
    u64* b = cv.take(M * K);
    fout[2 * j] = (u64*)A[j];
    fsum[2 * j] = a;
    fn[2 * j] = nx;
    frole[2 * j] = MPC_ROLE_TRIPLE_A;
    fout[2 * j + 1] = (u64*)B[j];
    fsum[2 * j + 1] = b;
    fn[2 * j + 1] = M * K;
    frole[2 * j + 1] = MPC_ROLE_TRIPLE_B;
    fop[2 * j] = fop[2 * j + 1] = op_ids[j];
    cg[j].d = d[j];
    cg[j].ho = tb.ho;
    cg[j].wo = tb.wo;
    cg[j].src2[0] = a;
    g.jobs[j] = GemmJob{b, nullptr, nullptr, nullptr, nullptr, (u64*)C[j] + (i64)(P - 1) * M * N};
    // every job's K range is split the same number of ways: at most its sub-steps
    g.max_splits = std::min<int>(g.max_splits, (int)ceil_div(K, 16));
  }
  for (int q = 0; q < 2 * count; ++q)
    if (int rc = launch_fill_sum(P, fn[q], seed, fop[q], frole[q], fout[q], fsum[q], s)) return rc;
  GemmArgs used{};
  if (int rc = run_gemm(g, algo, cv.rest(), ws_bytes - cv.off, s, &used)) return rc;
  u64* Cs[MPC_MAX_TRIPLE_BATCH];
  u64 ops[MPC_MAX_TRIPLE_BATCH];
  for (int j = 0; j < count; ++j) {
    Cs[j] = (u64*)C[j];
    ops[j] = op_ids[j];
  }
  return share_products(P, used, seed, ops, Cs, s);
}

}  // extern "C"
