/*
 * mpc_ring.h - C ABI of the B300 (sm_103a) private ring linear-algebra library.
 *
 * The library implements the hot path of CrypTen's secure multi-party
 * computation (arXiv 2109.00984): additive secret shares over the ring
 * Z/2^64 with fixed-point encoding (§5.1), Beaver-triple products for
 * elementwise / matmul / conv (§5.2, App. D.1.1), two-party local truncation
 * (App. D.1.1), and the comparison behind private ReLU: A2B with a
 * carry-lookahead adder, the sign bit, single-bit B2A (Alg. 2) and a Beaver
 * product with the mask (§5.2 "Comparators", App. D.1.2-D.1.4).
 * All parties are simulated on one GPU; "opening" a masked value is a
 * device-local reduction over the party axis, fused into the consuming kernel.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: MPC_OK (0) or a negative mpc_status.  The message of the
 *    last failure on the calling thread is returned by mpc_last_error().
 *  - Validation happens on the host before anything is launched; a call that
 *    returns an error has launched nothing (except MPC_ECUDA, reported when a
 *    launch itself failed).
 *  - Ownership: the caller owns every buffer, including workspaces sized by
 *    the mpc_*_workspace_size() functions.  Unless an entry point says
 *    otherwise, the library never allocates or frees memory.
 *  - Pointers marked "device" must point to memory of the current CUDA
 *    device.  Nothing synchronises: every call is asynchronous on `stream`
 *    (a cudaStream_t passed as void*, NULL = legacy default stream), except
 *    mpc_sync_status().
 *  - Shares are uint64 words, party-major and C-contiguous: a tensor of
 *    shape S held by P parties is laid out as [P][S].  Public ring tensors
 *    are [S].  Ring arithmetic wraps modulo 2^64; s(.) is the two's-complement
 *    signed view.
 *  - Randomness is explicit.  Every random word is word j of a Philox4x64-10
 *    stream (Salmon et al., SC'11) with key (seed, 0) and counter
 *    (j / 4, op_id, (role << 32) | (sub << 8) | party, 0), output word j % 4.
 *    The roles are the MPC_ROLE_* values below.  Equal (seed, op_id) give
 *    bit-identical results; callers must not reuse an op_id for two pieces
 *    of material.
 *  - Errors found on the device (an out-of-range real in mpc_ring_share, a
 *    bounded wait that gave up) are recorded in a per-device status word and
 *    returned by the next mpc_sync_status().
 *  - Parties: 1 <= P <= MPC_MAX_PARTIES.  The binary-share calls (mpc_a2b,
 *    mpc_private_relu, mpc_ltz) need P >= 2: for P = 2 the two binary-shared
 *    words go through one carry-lookahead adder, for P = 3..8 through a tree
 *    of ceil(log2 P) adder levels (P - 1 adders).  The fused-dealer calls
 *    (mpc_private_relu_fused and the function approximations) take P = 2 only.
 */
#ifndef MPC_RING_H
#define MPC_RING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPC_MAX_PARTIES 8
#define MPC_KS_GATES 12 /* secret ANDs in one 64-bit Kogge-Stone adder */

typedef enum {
  MPC_OK = 0,
  MPC_EINVAL = -1,      /* bad argument: null pointer, size, party count ... */
  MPC_ERANGE = -2,      /* a real value does not fit the fixed-point range   */
  MPC_ENOMEM = -3,      /* caller-provided workspace too small               */
  MPC_ECUDA = -4,       /* a CUDA runtime call or kernel launch failed       */
  MPC_ETIMEOUT = -5,    /* a bounded device-side wait gave up                */
  MPC_EUNSUPPORTED = -6 /* valid request the library does not implement      */
} mpc_status;

/* Ring GEMM engines for matmul / conv. */
typedef enum {
  MPC_ALGO_PLAIN = 0, /* CUDA-core 64-bit multiply-add emulated on 32-bit IMAD */
  MPC_ALGO_LIMB = 1,  /* 8-bit limb split on tcgen05 tensor cores              */
  MPC_ALGO_AUTO = 2   /* library picks (LIMB where the shape allows)           */
} mpc_algo;

/* PRG stream roles (third counter word bits 32..63). */
enum {
  MPC_ROLE_ZERO_ARITH = 0, /* arithmetic zero-share                         */
  MPC_ROLE_ZERO_BIN = 1,   /* binary zero-share in A2B, sub = owner q       */
  MPC_ROLE_TRIPLE_A = 2,
  MPC_ROLE_TRIPLE_B = 3,
  MPC_ROLE_TRIPLE_C = 4,
  MPC_ROLE_AND_A = 5, /* sub = gate index */
  MPC_ROLE_AND_B = 6,
  MPC_ROLE_AND_C = 7,
  MPC_ROLE_B2A_R = 8, /* party = MPC_TTP_PARTY: the dealer's secret bit */
  MPC_ROLE_B2A_BIN = 9,
  MPC_ROLE_B2A_ARITH = 10,
  MPC_ROLE_TRUNC_R = 11 /* Alg. 1 mask r (sub 0) and theta_r shares (sub 1) */
};
#define MPC_TTP_PARTY 255

/* Convolution geometry (NCHW data, OIHW weights, cross-correlation, zero
 * padding, groups = 1, dilation = 1).  A 1-D convolution is H = 1, kh = 1,
 * pad_h = 0. */
typedef struct {
  int64_t batch, c_in, h, w;  /* data  [batch][c_in][h][w]     */
  int64_t c_out, kh, kw;      /* weight [c_out][c_in][kh][kw]  */
  int64_t stride_h, stride_w; /* >= 1                          */
  int64_t pad_h, pad_w;       /* >= 0                          */
} mpc_conv_desc;

/* Counters of the protocol's communication, accumulated per process.
 * Rounds follow Table 3 of the paper: multiplication 1, AND 1, two-party
 * truncation 0, A2B 7 (one generate round + log2(64) prefix rounds), B2A 1. */
typedef struct {
  uint64_t calls;
  uint64_t rounds;              /* sequential opening rounds                */
  uint64_t bytes_opened;        /* bytes each party broadcasts               */
  uint64_t and_gates;           /* secret 64-bit AND word-gates evaluated    */
  uint64_t triple_words;        /* dealer words consumed by online calls     */
  uint64_t ring_macs;           /* multiply-adds in ring GEMMs (all parties) */
  uint64_t launches;            /* kernels launched by the library           */
} mpc_stats_t;

/* ---- status / diagnostics ------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none). */
const char* mpc_last_error(void);

/* Synchronises `stream`, then returns and clears the current device's
 * device-side status word (MPC_OK, MPC_ERANGE or MPC_ETIMEOUT), or MPC_ECUDA
 * if the stream reports an error. */
int mpc_sync_status(void* stream);

/* Copies the accumulated counters; mpc_reset_stats() zeroes them. */
int mpc_get_stats(mpc_stats_t* out);
int mpc_reset_stats(void);

/* Per-kernel timing.  While enabled, each launch of a timed kernel is
 * bracketed by two CUDA events on its stream (no synchronisation).
 * mpc_profile_read() waits for those events and returns, for the kernel
 * `kernel` ("gemm_plain", "gemm_plain_batched", "gemm_limb", "limb_planes",
 * "batched_open", "private_relu", "private_relu_fused", "beaver_mul", "a2b"),
 * the number of launches and their summed device time
 * since the last mpc_profile_reset().  Not for use inside stream capture. */
int mpc_profile_enable(int on);
int mpc_profile_reset(void);
int mpc_profile_read(const char* kernel, uint64_t* launches, double* total_ms);
/* The union of the intervals of those launches (ms): the time during which
 * at least one launch of `kernel` was running on any stream.  Launches that
 * overlap (e.g. the same kernel on a dealer stream and the main stream) count
 * once, so work / busy time is the kernel's throughput while it runs. */
int mpc_profile_busy(const char* kernel, double* busy_ms);

/* Diagnostic of the bounded-wait status path (the paper has no counterpart:
 * it concerns this library's device-side failure reporting).  Launches one
 * warp on `stream` whose thread 0 waits for an mbarrier phase that never
 * completes, through the same bounded wait and abort flag the limb engine's
 * roles use, but with a limit of limit_ns (1 us .. 1 s) instead of 2 s.  When
 * the limit passes it records MPC_ETIMEOUT in the device status word and the
 * kernel returns; nothing else is in flight, so the context stays usable.  The
 * next mpc_sync_status() returns MPC_ETIMEOUT (and clears it).  A limb-engine
 * launch made while the status word still holds MPC_ETIMEOUT gives up at its
 * first wait that does not complete at once, so read the status first. */
int mpc_test_wait_timeout(int64_t limit_ns, void* stream);

/* ---- sharing / reveal (§5.1, App. D.1.1) --------------------------------- */

/* Encode and share reals.  x: device double[n].  shares: device u64 [P][n].
 * x_enc = rint(x * 2^frac_bits) (ties to even); R_p = stream(ZERO_ARITH,
 * party p); shares[p] = R_p - R_{(p-1) mod P} + (p == src ? x_enc : 0).
 * |x * 2^frac_bits| >= 2^63 or a non-finite x stores 0 for that element and
 * records MPC_ERANGE for mpc_sync_status().  0 <= frac_bits <= 62. */
int mpc_ring_share(const double* x, int64_t n, int P, int src, int frac_bits, uint64_t seed,
                   uint64_t op_id, uint64_t* shares, void* stream);

/* Share ring elements that are already encoded: as mpc_ring_share without
 * the encoding step.  x_ring: device u64[n]. */
int mpc_ring_share_encoded(const uint64_t* x_ring, int64_t n, int P, int src, uint64_t seed,
                           uint64_t op_id, uint64_t* shares, void* stream);

/* Open shares: ring_out[i] = sum_p shares[p][i] (mod 2^64) and/or
 * real_out[i] = (double)s(ring value) / 2^frac_bits.  Either output may be
 * NULL, not both.  All pointers device. */
int mpc_reveal(const uint64_t* shares, int P, int64_t n, int frac_bits, uint64_t* ring_out,
               double* real_out, void* stream);

/* ---- dealer / trusted third party (§4, App. D.1.1-D.1.3) ----------------- */

/* Elementwise Beaver triple: A, B, C device u64 [P][n]; A[p] = stream(TRIPLE_A,
 * p), B[p] = stream(TRIPLE_B, p), c = (sum A)(sum B), C[p] = stream(TRIPLE_C, p)
 * for p < P-1 and C[P-1] = c - sum_{p<P-1} C[p]. */
int mpc_ttp_mul_triple(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* A,
                       uint64_t* B, uint64_t* C, void* stream);

/* Matmul triple: A [P][M][K], B [P][K][N], C [P][M][N] (device), c = a b, the
 * streams and the correction as for mpc_ttp_mul_triple (word index = flat
 * element index).  ws: device workspace of mpc_matmul_triple_workspace_size()
 * bytes.  algo selects the ring GEMM engine for c. */
size_t mpc_matmul_triple_workspace_size(int P, int64_t M, int64_t N, int64_t K, int algo);
int mpc_ttp_matmul_triple(int P, int64_t M, int64_t N, int64_t K, uint64_t seed,
                          uint64_t op_id, uint64_t* A, uint64_t* B, uint64_t* C, int algo,
                          void* ws, size_t ws_bytes, void* stream);

/* Convolution triple: A data-shaped [P][batch][c_in][h][w], B weight-shaped
 * [P][c_out][c_in][kh][kw], C output-shaped [P][batch][c_out][ho][wo], with
 * c = conv2d(a, b) over the ring. */
size_t mpc_conv2d_triple_workspace_size(int P, const mpc_conv_desc* d, int algo);
int mpc_ttp_conv2d_triple(int P, const mpc_conv_desc* d, uint64_t seed, uint64_t op_id,
                          uint64_t* A, uint64_t* B, uint64_t* C, int algo, void* ws,
                          size_t ws_bytes, void* stream);

/* A batch of `count` (1 <= count <= MPC_MAX_TRIPLE_BATCH) convolution triples,
 * triple j of descriptor d[j] dealt at op id op_ids[j] into the caller's
 * A[j], B[j], C[j] (device, shaped as for mpc_ttp_conv2d_triple): word for
 * word what `count` calls of mpc_ttp_conv2d_triple give (the dealer's role
 * in the paper's offline phase, §4).  Every d[j] must have d[0]'s output
 * shape (c_out, batch, ho, wo); c_in, h, w, the kernel, stride and padding
 * may differ.  On the limb engine the count products c_j = conv(a_j, b_j)
 * run as the jobs of one GEMM launch (each with its own K, split alike)
 * after one digit-plane launch per run of equal descriptors; on the plain
 * engine the triples are dealt in turn.  d, op_ids, A, B and C are host
 * arrays of count entries.  ws: device workspace of
 * mpc_conv2d_triples_workspace_size() bytes (0 for invalid arguments).
 * Errors: MPC_EINVAL (party count, count, a descriptor, output shapes that
 * differ, null pointers), MPC_ENOMEM (workspace), MPC_EUNSUPPORTED (shape
 * outside the limb engine). */
#define MPC_MAX_TRIPLE_BATCH 8
size_t mpc_conv2d_triples_workspace_size(int P, int count, const mpc_conv_desc* d, int algo);
int mpc_ttp_conv2d_triples(int P, int count, const mpc_conv_desc* d, uint64_t seed,
                           const uint64_t* op_ids, uint64_t* const* A, uint64_t* const* B,
                           uint64_t* const* C, int algo, void* ws, size_t ws_bytes,
                           void* stream);

/* Binary AND triples for `gates` gates over n words: T device u64
 * [gates][3][P][n] holding (a, b, c) per gate, a and b from the AND_A/AND_B
 * streams (sub = gate), c = (xor_p a_p) & (xor_p b_p) shared with AND_C
 * words for p < P-1 and the XOR correction on party P-1. */
int mpc_ttp_and_triples(int P, int64_t n, int gates, uint64_t seed, uint64_t op_id,
                        uint64_t* T, void* stream);

/* Random-bit pairs for B2A (App. D.1.3, Alg. 2): r = bit 0 of
 * stream(B2A_R, party MPC_TTP_PARTY); r_arith device u64 [P][n] with
 * r_arith[p] = stream(B2A_ARITH, p) for p < P-1 and r - sum on P-1;
 * r_bin device u64 [P][(n + 63) / 64], bit (i % 64) of word i / 64 of party
 * p = bit 0 of stream(B2A_BIN, p) word i for p < P-1, XOR-corrected on P-1.
 * Unused tail bits of r_bin are 0. */
int mpc_ttp_b2a_bits(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* r_arith,
                     uint64_t* r_bin, void* stream);

/* ---- online arithmetic (§5.2, App. D.1.1) -------------------------------- */

/* Fused elementwise Beaver product: one pass reads X, Y, A, B, C (device u64
 * [P][n]), opens E = sum_p (X_p - A_p) and F = sum_p (Y_p - B_p) in
 * registers, and writes Z_p = C_p + E B_p + A_p F (+ E F on party 0), then,
 * if trunc_bits > 0, Z_p = s(Z_p) >> trunc_bits (two-party local
 * truncation).  E_out / F_out (device u64[n]) receive the opened values when
 * not NULL.  Z may alias X or Y. */
int mpc_beaver_mul(int P, int64_t n, const uint64_t* X, const uint64_t* Y, const uint64_t* A,
                   const uint64_t* B, const uint64_t* C, uint64_t* Z, uint64_t* E_out,
                   uint64_t* F_out, int trunc_bits, void* stream);

/* Beaver matmul: X [P][M][K], Y [P][K][N], triple A [P][M][K], B [P][K][N],
 * C [P][M][N], Z [P][M][N] (device).  Z_p = C_p + E B_p + A_p F (+ E F on
 * party 0) with E = sum(X - A), F = sum(Y - B), optionally truncated by
 * trunc_bits.  ws: device workspace of mpc_matmul_workspace_size() bytes.
 * K = 0 gives Z = C (truncated); X, Y, A, B are then empty and may be NULL.
 * Each of M*K, K*N and M*N must be at most 2^52 words (MPC_EUNSUPPORTED
 * otherwise; the workspace-size functions return 0 for such shapes). */
size_t mpc_matmul_workspace_size(int P, int64_t M, int64_t N, int64_t K, int algo);
int mpc_beaver_matmul(int P, int64_t M, int64_t N, int64_t K, const uint64_t* X,
                      const uint64_t* Y, const uint64_t* A, const uint64_t* B,
                      const uint64_t* C, uint64_t* Z, int algo, int trunc_bits, void* ws,
                      size_t ws_bytes, void* stream);

/* Beaver convolution (App. D.1.1: the identity holds for any bilinear f):
 * X data [P][batch][c_in][h][w], W weights [P][c_out][c_in][kh][kw], triple
 * A (data-shaped), B (weight-shaped), C (output-shaped), Z output
 * [P][batch][c_out][ho][wo]; all device. */
size_t mpc_conv2d_workspace_size(int P, const mpc_conv_desc* d, int algo);
int mpc_beaver_conv2d(int P, const mpc_conv_desc* d, const uint64_t* X, const uint64_t* W,
                      const uint64_t* A, const uint64_t* B, const uint64_t* C, uint64_t* Z,
                      int algo, int trunc_bits, void* ws, size_t ws_bytes, void* stream);

/* Beaver convolution followed by the fused private ReLU, two parties (§5.2
 * "Comparators", App. D.1.1, D.1.4): the same result as
 *   mpc_beaver_conv2d(2, d, X, W, A, B, C, Z, algo, trunc_bits, ws, ...) then
 *   mpc_private_relu_fused(2, n, Z, Y, seed, relu_op, ...)
 * bit for bit (material at relu_op .. relu_op + 3), with Y in place of Z.  When
 * the convolution's GEMM is split along K, the ReLU kernel adds the partial
 * sums, C and the truncation itself as it loads each element, instead of a
 * separate reduction kernel writing Z first.  Y [2][batch][c_out][ho][wo]
 * (device); ws as mpc_conv2d_workspace_size().  P must be 2. */
int mpc_beaver_conv2d_relu(int P, const mpc_conv_desc* d, const uint64_t* X, const uint64_t* W,
                           const uint64_t* A, const uint64_t* B, const uint64_t* C, uint64_t* Y,
                           int algo, int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                           size_t ws_bytes, void* stream);

/* Input-independent half of a Beaver convolution on the limb engine (App.
 * D.1.1: F = W - B does not depend on the data, so it can be opened as soon as
 * the triple is dealt; the regrouping of the product is the one of
 * mpc_beaver_conv2d).  Opens F = sum_p (W_p - B_p) and cuts into prep the
 * digit planes of G = B_0 + F, B_1 .. B_{P-1}, F and of im2col(A_p) for every
 * party (the GEMM operands that do not involve X).  W, A, B as for
 * mpc_beaver_conv2d (device, read only); prep: caller-owned device buffer of
 * mpc_conv2d_prep_size() bytes (0 = shape or party count not supported: the
 * limb engine's shape limits), written, read by the prepared call below.
 * Counts one round and the F bytes opened.  MPC_ENOMEM if prep_bytes is too
 * small; no workspace. */
size_t mpc_conv2d_prep_size(int P, const mpc_conv_desc* d);
int mpc_beaver_conv2d_prepare(int P, const mpc_conv_desc* d, const uint64_t* W, const uint64_t* A,
                              const uint64_t* B, void* prep, size_t prep_bytes, void* stream);

/* The data-dependent half: opens E = sum_p (X_p - A_p), gathers im2col(E) into
 * digit planes and runs the limb-engine GEMM on them and the prepared planes
 * (the same triple A as the prepare call).  Results equal mpc_beaver_conv2d /
 * mpc_beaver_conv2d_relu with algo = MPC_ALGO_LIMB bit for bit.  ws as
 * mpc_conv2d_workspace_size(P, d, MPC_ALGO_LIMB).  The ReLU variant needs
 * P = 2 (material at relu_op .. relu_op + 3). */
int mpc_beaver_conv2d_prepared(int P, const mpc_conv_desc* d, const uint64_t* X,
                               const uint64_t* A, const uint64_t* C, const void* prep,
                               size_t prep_bytes, uint64_t* Z, int trunc_bits, void* ws,
                               size_t ws_bytes, void* stream);
int mpc_beaver_conv2d_relu_prepared(int P, const mpc_conv_desc* d, const uint64_t* X,
                                    const uint64_t* A, const uint64_t* C, const void* prep,
                                    size_t prep_bytes, uint64_t* Y, int trunc_bits, uint64_t seed,
                                    uint64_t relu_op, void* ws, size_t ws_bytes, void* stream);

/* Beaver convolution, a residual sum and the fused ReLU, two parties (a
 * ResNet block's second convolution, its shortcut and its ReLU): Y =
 * ReLU(trunc(conv) + S) with the words of mpc_beaver_conv2d (or _prepared)
 * followed by mpc_private_relu_fused_add(2, n, Z, S, Y, seed, relu_op); the
 * ReLU kernel adds the split-K partial sums, C, the truncation and S as it
 * loads each element.  S device u64 [2][batch][c_out][ho][wo]; Y must not
 * alias S.  Arguments otherwise as mpc_beaver_conv2d_relu and
 * mpc_beaver_conv2d_relu_prepared. */
int mpc_beaver_conv2d_relu_add(int P, const mpc_conv_desc* d, const uint64_t* X,
                               const uint64_t* W, const uint64_t* A, const uint64_t* B,
                               const uint64_t* C, const uint64_t* S, uint64_t* Y, int algo,
                               int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                               size_t ws_bytes, void* stream);
int mpc_beaver_conv2d_relu_prepared_add(int P, const mpc_conv_desc* d, const uint64_t* X,
                                        const uint64_t* A, const uint64_t* C, const void* prep,
                                        size_t prep_bytes, const uint64_t* S, uint64_t* Y,
                                        int trunc_bits, uint64_t seed, uint64_t relu_op, void* ws,
                                        size_t ws_bytes, void* stream);

/* Prepared products (limb engine): the preparation goes one step further and
 * also computes each party's input-independent product, C'_p = C_p + A_p F
 * with F = W - B opened (App. D.1.1: Z_p = C_p + E B_p + A_p F + [p = 0] E F),
 * so the online half is one operand pair per party, Z_p = C'_p + E G_p with
 * G_0 = B_0 + F and G_p = B_p.  prep (device, mpc_conv2d_prep_products_size
 * bytes) receives the digit planes of G_0 .. G_{P-1} and C'_0 .. C'_{P-1};
 * the preparation uses ws (mpc_conv2d_prepare_products_workspace_size bytes).
 * The online calls read neither W, B nor C, and give the words of
 * mpc_beaver_conv2d / mpc_beaver_conv2d_relu with the same triple (ws as
 * mpc_conv2d_workspace_size(P, d, MPC_ALGO_LIMB)).  The sizes are 0 for
 * invalid arguments or shapes outside the limb engine. */
size_t mpc_conv2d_prep_products_size(int P, const mpc_conv_desc* d);
size_t mpc_conv2d_prepare_products_workspace_size(int P, const mpc_conv_desc* d);
int mpc_beaver_conv2d_prepare_products(int P, const mpc_conv_desc* d, const uint64_t* W,
                                       const uint64_t* A, const uint64_t* B, const uint64_t* C,
                                       void* prep, size_t prep_bytes, void* ws, size_t ws_bytes,
                                       void* stream);
int mpc_beaver_conv2d_prepared_products(int P, const mpc_conv_desc* d, const uint64_t* X,
                                        const uint64_t* A, const void* prep, size_t prep_bytes,
                                        uint64_t* Z, int trunc_bits, void* ws, size_t ws_bytes,
                                        void* stream);
int mpc_beaver_conv2d_relu_prepared_products(int P, const mpc_conv_desc* d, const uint64_t* X,
                                             const uint64_t* A, const void* prep,
                                             size_t prep_bytes, uint64_t* Y, int trunc_bits,
                                             uint64_t seed, uint64_t relu_op, void* ws,
                                             size_t ws_bytes, void* stream);

/* Beaver matmul that allocates nothing (the paper has no counterpart: this is
 * an interface for callers that can neither allocate device memory when they
 * call the library nor hand it a workspace, e.g. a host program whose device
 * memory is wholly reserved by another framework's pool, or code running where
 * allocation calls are not allowed).  Same arguments, layouts and results as
 * mpc_beaver_matmul with the plain engine, minus algo/ws.  Its scratch,
 * M*K + 2*K*N words (each region rounded up to 32 words), lives in a fixed
 * library-owned device array of MPC_NOALLOC_SCRATCH_WORDS words (8 MiB),
 * present on every device that loads the library until the process exits;
 * larger requests return MPC_ENOMEM and launch nothing (the dimensions are
 * bounded against the array before any product of them is formed, so no
 * shape can wrap the size check).  Its protocol counters are those of
 * mpc_beaver_matmul.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.  The first call on a
 * device looks up the array's device address (with that device current), so
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (each call writes every word it reads
 * before reading it); calls whose kernels overlap on the GPU race on it, so
 * serialise them. */
#define MPC_NOALLOC_SCRATCH_WORDS (1ll << 20)
int mpc_beaver_matmul_noalloc(int P, int64_t M, int64_t N, int64_t K, const uint64_t* X,
                              const uint64_t* Y, const uint64_t* A, const uint64_t* B,
                              const uint64_t* C, uint64_t* Z, int trunc_bits, void* stream);

/* ---- batched Beaver matmul ----------------------------------------------- */

/* One product of a batch: X [P][M][K], Y [P][K][N], triple A [P][M][K],
 * B [P][K][N], C [P][M][N] and output Z [P][M][N], all device pointers. */
typedef struct {
  int64_t M, N, K;
  const uint64_t* X;
  const uint64_t* Y;
  const uint64_t* A;
  const uint64_t* B;
  const uint64_t* C;
  uint64_t* Z;
} mpc_matmul_desc;

/* Tuning of the batched call: products with M*N*K >= limb_min_macs run on the
 * limb engine (algo AUTO); persistent_ctas = CTAs of the persistent plain
 * kernel, limb_ctas = CTAs of the persistent limb kernel (0 = one per SM). */
typedef struct {
  double limb_min_macs;
  int persistent_ctas;
  int limb_ctas;
} mpc_tune;

/* Fills the built-in tuning (limb from 2^24 ring MACs up). */
int mpc_tune_default(mpc_tune* out);

/* Batched Beaver matmul (App. D.1.1 applied to many products at once): every
 * product is opened in one pass (one round for the whole batch), then the
 * products below the limb threshold run in one persistent launch of the plain
 * engine that hands out output tiles of any product from an atomic counter
 * (largest K first), and the others in one persistent launch of the limb
 * engine (after one digit-plane launch for all of them) that hands out 128 x
 * 128 tiles of any product and party the same way.  Results equal
 * mpc_beaver_matmul on each product.  descs: host array of `count`
 * descriptors (read during the call only).  tune may be NULL (defaults).
 * ws: device workspace of mpc_matmul_batched_workspace_size() bytes (it holds
 * the work tables, every product's opened E, F and B_0 + F, and the digit
 * planes of every limb product).  Stream-capturable: the descriptors and the
 * limb engine's tensor maps reach the device as kernel parameters. */
size_t mpc_matmul_batched_workspace_size(int P, int count, const mpc_matmul_desc* descs, int algo,
                                         const mpc_tune* tune);
int mpc_beaver_matmul_batched(int P, int count, const mpc_matmul_desc* descs, int algo,
                              const mpc_tune* tune, int trunc_bits, void* ws, size_t ws_bytes,
                              void* stream);

/* Autotuner: times the batched call (algo AUTO) for limb thresholds from
 * "never" through 2^32 .. 2^16 ring MACs to "always" (each candidate the
 * fastest of four calls after one warm-up, with L2 evicted before each call by
 * overwriting up to 256 MB of ws, and device time only: each timed call waits
 * behind a 20 ms device delay while the host enqueues it) and returns the
 * fastest in *out.
 * Synchronises `stream`; not for use inside stream capture.  Writes Z. */
int mpc_autotune_batched(int P, int count, const mpc_matmul_desc* descs, int trunc_bits,
                         void* ws, size_t ws_bytes, void* stream, mpc_tune* out);

/* Plain ring GEMM Z = C + A B over Z/2^64: A [M][K], B [K][N], C [M][N] or
 * NULL, Z [M][N] (device, row-major).  ws as mpc_ring_gemm_workspace_size(). */
size_t mpc_ring_gemm_workspace_size(int64_t M, int64_t N, int64_t K, int algo);
int mpc_ring_gemm(int64_t M, int64_t N, int64_t K, const uint64_t* A, const uint64_t* B,
                  const uint64_t* C, uint64_t* Z, int algo, void* ws, size_t ws_bytes,
                  void* stream);

/* Two-party local truncation (App. D.1.1), in place on device u64 [P][n]:
 * share = floor(s(share) / l) with l = divisor if divisor > 0, else
 * 2^frac_bits (an arithmetic shift).  0 <= frac_bits <= 63. */
int mpc_truncate(int P, int64_t n, uint64_t* shares, int frac_bits, int64_t divisor,
                 void* stream);

/* Truncation for any number of parties, Alg. 1 (wrap count), in place on
 * device u64 [P][n]: every quantity in the signed view, so that
 * x = sum_p s(x_p) - theta_x 2^64; the parties open z = x + r (one round),
 * [theta_x] = theta_z + [beta] - [theta_r] (eta = 0, as in the paper) and
 * party p keeps floor(s(x_p) / 2^f) - [theta_x]_p 2^(64-f).  The result is
 * within P units of floor(x / 2^f) except when the signed sum x + r
 * overflows (probability about |x| / 2^64).  r, theta_r: [P][n] from
 * mpc_ttp_trunc_pairs.  1 <= frac_bits <= 63. */
int mpc_truncate_nparty(int P, int64_t n, uint64_t* shares, const uint64_t* r,
                        const uint64_t* theta_r, int frac_bits, void* stream);

/* Dealer material for Alg. 1: r [P][n] with r[p] = stream(TRUNC_R, sub 0, p),
 * and theta_r [P][n], shares of the signed wrap count of r's shares:
 * theta_r[p] = stream(TRUNC_R, sub 1, p) for p < P-1, correction on P-1. */
int mpc_ttp_trunc_pairs(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* r,
                        uint64_t* theta_r, void* stream);

/* Beaver square (App. D.1.1 "Square"): with a pair ([a], [b]), b = a^2, open
 * eps = sum_p (X_p - A_p) in registers and write Z_p = B_p + 2 eps A_p
 * (+ eps^2 on party 0), then optionally s(Z_p) >> trunc_bits.  One round.
 * X, A, B, Z device u64 [P][n]; Z may alias X. */
int mpc_beaver_square(int P, int64_t n, const uint64_t* X, const uint64_t* A, const uint64_t* B,
                      uint64_t* Z, int trunc_bits, void* stream);

/* Dealer pair for mpc_beaver_square: A[p] = stream(TRIPLE_A, p), b = a^2
 * shared as B[p] = stream(TRIPLE_C, p) for p < P-1 and the correction on P-1. */
int mpc_ttp_square_pair(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* A, uint64_t* B,
                        void* stream);

/* [x < 0] (§5.2 "Comparators"): B2A(MSB(A2B([x]))) as arithmetic shares of an
 * unscaled 0/1 bit, Out device u64 [P][n].  Material as for mpc_private_relu
 * without the elementwise triple: and_triples [12 (P-1)][3][P][n], r_arith,
 * r_bin from mpc_ttp_b2a_bits; (seed, op_id) drive the A2B masks.  The other
 * comparators follow: [x < y] = [x - y < 0], [x > y] = [y - x < 0],
 * [x >= y] = 1 - [x < y], [x <= y] = 1 - [x > y], [x == y] = [x <= y] - [x < y]. */
int mpc_ltz(int P, int64_t n, const uint64_t* X, uint64_t* out, const uint64_t* and_triples,
            const uint64_t* r_arith, const uint64_t* r_bin, uint64_t seed, uint64_t op_id,
            void* stream);

/* Public affine map, local (§5.2): Z_p = scale * X_p, plus `offset` (a public
 * ring element) on party 0, then if trunc_bits > 0 the two-party local
 * truncation s(Z_p) >> trunc_bits.  Z may alias X. */
int mpc_affine(int P, int64_t n, const uint64_t* X, uint64_t* Z, int64_t scale, uint64_t offset,
               int trunc_bits, void* stream);

/* ---- local share operations (no communication) --------------------------- */

/* Private addition / subtraction (§5.2 "Private addition"): Z_p = X_p + Y_p
 * (or X_p - Y_p) for every party.  Each array holds party p's n words at
 * p * pstride (0 means n, i.e. the contiguous [P][n] layout), so strided
 * party slices of a larger tensor can be used directly.  Z may alias X or Y. */
int mpc_add(int P, int64_t n, const uint64_t* X, int64_t x_pstride, const uint64_t* Y,
            int64_t y_pstride, uint64_t* Z, int64_t z_pstride, void* stream);
int mpc_sub(int P, int64_t n, const uint64_t* X, int64_t x_pstride, const uint64_t* Y,
            int64_t y_pstride, uint64_t* Z, int64_t z_pstride, void* stream);

/* Window taps for pooling (a layout operation, no arithmetic): X shares
 * [P][batch][c_in][h][w] -> taps [kh*kw][P][batch][c_in][ho][wo], tap
 * t = r * kw + s holding X at (oh * stride_h + r - pad_h, ow * stride_w + s -
 * pad_w), zero outside.  Uses batch, c_in, h, w, kh, kw, strides and pads of
 * the descriptor (c_out is ignored).  A 3x3 max pool is then a tree of
 * max(a, b) = b + ReLU(a - b) over the taps. */
int mpc_window_taps(int P, const mpc_conv_desc* d, const uint64_t* X, uint64_t* taps,
                    void* stream);

/* Global average pooling: out[p][r] = floor(s(sum_{j<hw} X[p][r*hw + j]) / hw),
 * a local sum followed by two-party truncation by the public window size
 * (App. D.1.1).  X [P][rows][hw], out [P][rows]. */
int mpc_global_avgpool(int P, int64_t rows, int64_t hw, const uint64_t* X, uint64_t* out,
                       void* stream);

/* ---- binary shares and comparison (§5.1-5.2, App. D.1.2-D.1.4) ---------- */

/* A2B (§5.1, App. D.1.3) for P = 2..8: arith [P][n] -> binary [P][n]
 * (device).  Each party's share y_q is binary-shared with the ZERO_BIN stream
 * (sub = q): party p holds M_{q,p} ^ M_{q,(p-1) mod P} ^ (p == q ? y_q : 0).
 * P = 2: the two binary-shared words are added by one 64-bit Kogge-Stone
 * adder whose 12 secret ANDs use and_triples [12][3][2][n]
 * (mpc_ttp_and_triples) in the order: generate, then for d = 1, 2, 4, 8, 16,
 * 32 the G-update and (d < 32) the P-update.  P = 3..8: a tree of adders;
 * each level adds neighbours (0, 1), (2, 3), ... and passes an odd last
 * addend up; adder a (numbered level by level, left to right) uses gates
 * 12a .. 12a + 11 of and_triples [12 (P-1)][3][P][n].  7 rounds per level.
 * P = 1 returns MPC_EUNSUPPORTED. */
int mpc_a2b(int P, int64_t n, const uint64_t* arith, uint64_t* binary,
            const uint64_t* and_triples, uint64_t seed, uint64_t op_id, void* stream);

/* Private ReLU for P = 2..8 in one kernel: [x > 0] = B2A(MSB(A2B(-x)))
 * (comparator of §5.2, Alg. 2), then Y = Beaver product of X with the 0/1
 * mask (not truncated).  X, Y device u64 [P][n] (may alias); and_triples
 * [12 (P-1)][3][P][n] (the adder or adder tree of mpc_a2b); r_arith [P][n]
 * and r_bin [P][(n+63)/64] from mpc_ttp_b2a_bits; mul_A, mul_B, mul_C
 * [P][n] each, the elementwise triple from mpc_ttp_mul_triple.  (seed,
 * op_id) drive the A2B binary zero-shares.  P = 1 returns MPC_EUNSUPPORTED. */
int mpc_private_relu(int P, int64_t n, const uint64_t* X, uint64_t* Y,
                     const uint64_t* and_triples, const uint64_t* r_arith,
                     const uint64_t* r_bin, const uint64_t* mul_A, const uint64_t* mul_B,
                     const uint64_t* mul_C, uint64_t seed, uint64_t op_id, void* stream);

/* Private ReLU with the dealer fused in (P = 2): the same result as
 *   mpc_ttp_and_triples(2, n, 12, seed, op_id) -> T,
 *   mpc_ttp_b2a_bits(2, n, seed, op_id + 1) -> r_arith, r_bin,
 *   mpc_ttp_mul_triple(2, n, seed, op_id + 2) -> A, B, C,
 *   mpc_private_relu(2, n, X, Y, T, r_arith, r_bin, A, B, C, seed, op_id + 3),
 * bit for bit, but every piece of dealer material is regenerated in registers
 * from its Philox stream instead of being written to and read from memory
 * (the trusted dealer and both parties are simulated in one kernel).  X, Y
 * device u64 [2][n] (may alias).  Uses op ids op_id .. op_id + 3. */
int mpc_private_relu_fused(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                           uint64_t op_id, void* stream);

/* mpc_private_relu_fused of X + S (§5.2 "Private addition" then the ReLU): the
 * same words as mpc_add(2, n, X, 0, S, 0, T, 0) followed by
 * mpc_private_relu_fused(2, n, T, Y, seed, op_id), with the local addition
 * folded into the ReLU
 * kernel's load (a residual connection's sum goes straight into its ReLU).
 * S device u64 [2][n] or null (then exactly mpc_private_relu_fused); Y may
 * alias X or S.  Errors as mpc_private_relu_fused. */
int mpc_private_relu_fused_add(int P, int64_t n, const uint64_t* X, const uint64_t* S,
                               uint64_t* Y, uint64_t seed, uint64_t op_id, void* stream);

/* Private maximum of two sharings, P = 2 (§5.2 "Comparators"; the step of a
 * max-pool tree): Y = B + ReLU(A - B), with the ReLU's dealer material that
 * mpc_private_relu_fused (op ids op_id .. op_id + 3) draws for elements
 * elem_offset .. elem_offset + n - 1 of a longer batch, so that the slices of
 * one batched comparison (pair i of a tree level at elem_offset = i n) give
 * the words of mpc_sub, one mpc_private_relu_fused over the whole batch and
 * mpc_add.  elem_offset a non-negative multiple of 4 (MPC_EINVAL otherwise).
 * A, B, Y device u64 [2][n]; Y may alias A or B.  The rounds of the batch are
 * counted once, by the slice at offset 0. */
int mpc_private_max_fused(int P, int64_t n, const uint64_t* A, const uint64_t* B, uint64_t* Y,
                          uint64_t seed, uint64_t op_id, int64_t elem_offset, void* stream);

/* ---- function approximations (App. D.2), two parties, fused dealer -------- */
/* Each call below evaluates one function elementwise on two-party shares of
 * fixed-point values (2^16) in ONE launch per element range: every dealer
 * word is regenerated from Philox in registers and every opening is a sum of
 * the two shares, so HBM traffic is X and Y only.  Step k of a function (a
 * Beaver product, a square, a comparison) draws its material at op id
 * op_id + 10 k, in the order the steps run.  X, Y: device u64 [2][n]; Y may
 * alias X (except for mpc_softmax).  P must be 2 (MPC_EUNSUPPORTED otherwise).
 * Products of two scaled values are followed by the two-party truncation by
 * 16 bits, so results carry a few ulps (2^-16) of error beyond the method's. */
#define MPC_APPROX_MAX_EXP_ITERS 20
#define MPC_APPROX_MAX_NR_ITERS 64

/* exp(x) by the limit approximation (1 + x / 2^iters)^(2^iters) (App. D.2.1):
 * a truncation by `iters` bits, then `iters` Beaver squarings (iters in
 * 1..20; 8 is the paper's default).  Accurate for x <~ 2^iters / 10; for
 * x < -2^iters the base turns negative. */
int mpc_exp(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int iters, void* stream);

/* 1/x by Newton-Raphson y <- y (2 - x y) (App. D.2.2), nr_iters iterations
 * from y0 = 3 exp(0.5 - x) + 0.003 (exp with exp_iters).  With all_positive
 * the input must be > 0; otherwise 1/x = sgn(x) / |x| with one comparison and
 * two more products.  Converges for 0 < x y0 < 2 (x up to ~ 200 by default). */
int mpc_reciprocal(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                   uint64_t op_id, int all_positive, int exp_iters, int nr_iters, void* stream);

/* sigmoid(x) (App. D.2.5): [x < 0] and |x| from one comparison and one product,
 * sigma(|x|) = 1 / (1 + exp(-|x|)) by Newton-Raphson from 0.75, then the
 * multiplexing product [x < 0] ? 1 - sigma(|x|) : sigma(|x|). */
int mpc_sigmoid(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
                int exp_iters, int nr_iters, void* stream);

/* tanh(x) = 2 sigmoid(2x) - 1 (App. D.2.5). */
int mpc_tanh(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
             int exp_iters, int nr_iters, void* stream);

/* erf(x) by the Maclaurin series 2/sqrt(pi) sum_{k=0}^{terms} (-1)^k
 * x^(2k+1) / (k! (2k+1)) (App. D.2.6; terms = 8 by default, at most 16):
 * one square, then `terms` products; poor for |x| > 1 as the paper notes. */
int mpc_erf(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int terms, void* stream);

/* x^(-1/2) for x > 0 by y <- y (3 - x y^2) / 2 (App. D.2.3), nr_iters
 * iterations from y0 = 3 g^16 + 0.3 g + 0.05 with g = exp(-x / 16) (the paper
 * gives no initial value; this one converges on [0.01, 100]).  mpc_sqrt
 * multiplies the result by x. */
int mpc_inv_sqrt(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                 uint64_t op_id, int exp_iters, int nr_iters, void* stream);
int mpc_sqrt(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
             int exp_iters, int nr_iters, void* stream);

/* ln(x) for x > 0 by Householder iterations (App. D.2.4): h = 1 - x exp(-y),
 * y <- y - sum_{k=1}^{order} h^k / k, `iters` iterations (default 3, order 8)
 * from y0 = x / 120 - 20 exp(-2x - 1) + 3.  With the limit approximation
 * inside, the iteration converges to 256 (1 - x^(-1/256)). */
int mpc_log(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed, uint64_t op_id,
            int exp_iters, int iters, int order, void* stream);

/* Maximum over the last axis (Table "max"/"argmax": tree reduction): X shares
 * [2][rows][m] -> out [2][rows].  Level l pairs adjacent elements,
 * max(a, b) = b + ReLU(a - b) with the ReLU of all pairs of the level at op id
 * op_id + 10 l (material indexed by the flat pair index row * floor(m'/2) + i);
 * an odd last element moves up unchanged.  Exact (no truncation).  workspace:
 * device, at least mpc_max_workspace_size bytes (none needed for m == 1). */
size_t mpc_max_workspace_size(int P, int64_t rows, int64_t m);
int mpc_max_lastdim(int P, int64_t rows, int64_t m, const uint64_t* X, uint64_t* out,
                    void* workspace, size_t ws_bytes, uint64_t seed, uint64_t op_id,
                    void* stream);

/* Softmax over the last axis (App. D.2, Table "softmax"): the max tree as in
 * mpc_max_lastdim, e = exp(x - max) with the next exp_iters op ids, s = sum of
 * e over the row (local), r = reciprocal(s) (positive form, s >= 1), then
 * Y = e * r with the elementwise triple at the next op id (flat index).
 * X, Y: device u64 [2][rows][m], Y must not alias X.  workspace: device, at
 * least mpc_softmax_workspace_size bytes.  Four to ceil(log2 m) + 4 launches. */
size_t mpc_softmax_workspace_size(int P, int64_t rows, int64_t m);
int mpc_softmax(int P, int64_t rows, int64_t m, const uint64_t* X, uint64_t* Y, void* workspace,
                size_t ws_bytes, uint64_t seed, uint64_t op_id, int exp_iters, int nr_iters,
                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPC_RING_H */
