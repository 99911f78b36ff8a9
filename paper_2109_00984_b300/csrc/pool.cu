// Local (communication-free) share operations used between the protocol's
// interactive steps: private addition / subtraction (§5.2 "Private
// addition"), the window-tap gather behind max pooling, and global average
// pooling as a local sum followed by two-party truncation by the public
// window size (App. D.1.1).
#include "common.cuh"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int kThreads = 256;

// Z_p = X_p (+/-) Y_p; party p's words start at p * stride in each array.
template <bool kSub>
__global__ void __launch_bounds__(kThreads) addsub_kernel(int P, i64 n, const u64* X, i64 xs,
                                                          const u64* Y, i64 ys, u64* Z, i64 zs) {
  const i64 total = (i64)P * n;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const i64 p = i / n, e = i % n;
    const u64 x = X[p * xs + e], y = Y[p * ys + e];
    Z[p * zs + e] = kSub ? x - y : x + y;
  }
}

// taps[t][p][b][c][oh][ow] = X[p][b][c][oh*sh + r - ph][ow*sw + s - pw] (0 outside),
// t = r * kw + s.  One thread per output position (b, c, oh, ow) writes all its
// taps for every party: the position is decoded once (three 64-bit divisions)
// instead of once per tap and party; the writes of consecutive threads stay
// consecutive within each (t, p) plane.
__global__ void __launch_bounds__(kThreads) taps_kernel(int P, mpc_conv_desc d, i64 ho, i64 wo,
                                                        const u64* __restrict__ X,
                                                        u64* __restrict__ taps) {
  const i64 nout = d.batch * d.c_in * ho * wo;
  const i64 nin = d.batch * d.c_in * d.h * d.w;
  const int kh = (int)d.kh, kw = (int)d.kw;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < nout;
       e += (i64)gridDim.x * blockDim.x) {
    const i64 ow = e % wo, q = e / wo;
    const i64 oh = q % ho, bc = q / ho;
    const i64 y0 = oh * d.stride_h - d.pad_h, x0 = ow * d.stride_w - d.pad_w;
    for (int r = 0; r < kh; ++r) {
      const i64 y = y0 + r;
      const bool yin = y >= 0 && y < d.h;
      for (int s = 0; s < kw; ++s) {
        const i64 x = x0 + s;
        const bool in = yin && x >= 0 && x < d.w;
        const i64 src = (bc * d.h + y) * d.w + x;
        u64* dst = taps + (i64)(r * kw + s) * P * nout + e;
        for (int p = 0; p < P; ++p) dst[(i64)p * nout] = in ? X[p * nin + src] : 0ull;
      }
    }
  }
}

// out[p][r] = floor(s(sum_j X[p][r * hw + j]) / hw).
__global__ void __launch_bounds__(kThreads) avgpool_kernel(int P, i64 rows, i64 hw,
                                                           const u64* __restrict__ X,
                                                           u64* __restrict__ out) {
  const i64 total = (i64)P * rows;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const u64* src = X + i * hw;
    u64 acc = 0;
    for (i64 j = 0; j < hw; ++j) acc += src[j];
    out[i] = floordiv_signed(acc, hw);
  }
}

template <bool kSub>
int addsub(int P, int64_t n, const uint64_t* X, int64_t xs, const uint64_t* Y, int64_t ys,
           uint64_t* Z, int64_t zs, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(xs >= 0 && ys >= 0 && zs >= 0, "negative party stride");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y && Z, "null pointer");
  if (xs == 0) xs = n;
  if (ys == 0) ys = n;
  if (zs == 0) zs = n;
  MPC_REQUIRE((P == 1 || (xs >= n && ys >= n && zs >= n)), "party stride shorter than n");
  addsub_kernel<kSub><<<grid_for((i64)P * n, kThreads), kThreads, 0, as_stream(stream)>>>(
      P, n, (const u64*)X, xs, (const u64*)Y, ys, (u64*)Z, zs);
  return check_launch(kSub ? "sub" : "add");
}

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_add(int P, int64_t n, const uint64_t* X, int64_t x_pstride, const uint64_t* Y,
            int64_t y_pstride, uint64_t* Z, int64_t z_pstride, void* stream) {
  return addsub<false>(P, n, X, x_pstride, Y, y_pstride, Z, z_pstride, stream);
}

int mpc_sub(int P, int64_t n, const uint64_t* X, int64_t x_pstride, const uint64_t* Y,
            int64_t y_pstride, uint64_t* Z, int64_t z_pstride, void* stream) {
  return addsub<true>(P, n, X, x_pstride, Y, y_pstride, Z, z_pstride, stream);
}

int mpc_window_taps(int P, const mpc_conv_desc* d, const uint64_t* X, uint64_t* taps,
                    void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(d != nullptr, "null descriptor");
  MPC_REQUIRE(d->batch >= 1 && d->c_in >= 1 && d->h >= 1 && d->w >= 1 && d->kh >= 1 &&
                  d->kw >= 1 && d->stride_h >= 1 && d->stride_w >= 1 && d->pad_h >= 0 &&
                  d->pad_w >= 0,
              "bad window geometry");
  MPC_REQUIRE(d->h + 2 * d->pad_h >= d->kh && d->w + 2 * d->pad_w >= d->kw,
              "window larger than the padded input");
  MPC_REQUIRE(X && taps, "null pointer");
  const i64 ho = (d->h + 2 * d->pad_h - d->kh) / d->stride_h + 1;
  const i64 wo = (d->w + 2 * d->pad_w - d->kw) / d->stride_w + 1;
  const i64 nout = d->batch * d->c_in * ho * wo;
  taps_kernel<<<grid_for(nout, kThreads), kThreads, 0, as_stream(stream)>>>(P, *d, ho, wo,
                                                                           (const u64*)X,
                                                                           (u64*)taps);
  return check_launch("window_taps");
}

int mpc_global_avgpool(int P, int64_t rows, int64_t hw, const uint64_t* X, uint64_t* out,
                       void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(rows >= 0 && hw >= 1, "bad pooling size");
  if (rows == 0) return MPC_OK;
  MPC_REQUIRE(X && out, "null pointer");
  avgpool_kernel<<<grid_for((i64)P * rows, kThreads), kThreads, 0, as_stream(stream)>>>(
      P, rows, hw, (const u64*)X, (u64*)out);
  return check_launch("global_avgpool");
}

}  // extern "C"
