// Internal declarations shared by the CUDA translation units of libdonof.
// Nothing here is part of the C ABI (include/donof.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/donof.h"

namespace donof {

// ---------------------------------------------------------------------------
// Device-resident header at the start of every workspace.
// ---------------------------------------------------------------------------
struct DevHeader {
  int32_t status;      // DONOF_OK or the first DONOF_ERR_* raised on the device
  int32_t e3;          // output exponent of the G split partials (0: true units)
  int32_t zero_exp;    // always 0 (epilogue exponent of raw partial sums)
  int32_t abort_flag;  // set when a bounded device wait gives up; cleared per build
  double E;            // energy of the last build
  double sC2;          // bound on ||C_act||_2^2 (Gershgorin on C_act^T C_act)
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
__host__ __device__ inline int round_up_int(int x, int a) { return (x + a - 1) / a * a; }

// Derived sizes of one problem.
struct Dims {
  int N, Q, A, Ap, Np, npair, ncwo, ng, pb, nblk, functional, layout, precision;
  int nsingle;  // singly occupied orbitals (Omega_I) at npair .. npair + nsingle - 1
  int splits;  // split-K factor of the G contraction (mixed path)
};

// Byte offsets of every buffer inside the workspace.
struct Layout {
  size_t header;
  // shared by both precisions
  size_t n, sqn, phi, dn, dsq, dphi, Acoef, Bcoef, Hd, hC, J, K, G, dEdg, Epart;
  size_t skp;  // deterministic split-K partials of the FP64 N x A products
  // FP64 path
  size_t X64, b64, Y64, Bun;
  // mixed path
  // integer + fraction planes (h, f) of the tensor-core operands and their per-row
  // exponents: B (Bhi/Blo, eB), C_act^T (Chi/Clo, eC), X^T for b (Xthi/Xtlo, eXt), X for G
  // (Xhi/Xlo, eX3 per split), Y (Yhi/Ylo, eY per split); the exponents of C^T and G^T for
  // lambda (eCf, eG; their planes share the buffers of h C_act below)
  size_t Bhi, Blo, eB, L1max, Chi, Clo, eC, cnorm, Xhi, Xlo, Xthi, Xtlo, eXt, b32, Yhi, Ylo,
      Gpart, D, rn2, spOf, eX3, eY, eCf, eG;
  // symmetric storage of the split B: per-AO scale exponents s, their source (max over P of
  // the row norms), per-slice maxima of the scaled row norms, and the split of
  // (diag 2^s C_act)^T that multiplies it
  size_t eS, rnmax, tmax, ChiS, CloS, eCs;
  size_t gram;  // per-chunk parts of the Gram matrix of C_act (fp32)
  // between the b and G contractions: w^P (fp32), per-split K and J partials (double),
  // fp32 copies of the J and K coefficient matrices ([Ap][Ap])
  size_t W, Ksp, Jsp, AcF, BcF;
  // h C_act and lambda = C^T G on the tensor cores: the split of h (then of C^T) extended
  // by its residual (four K-block planes per slot, hAH/hAF, exponents eh), the same planes
  // of C_act^T (then of G^T) (cPH/cPF), and the fp32 products of the four blocks (hpart)
  size_t hAH, hAF, cPH, cPF, eh, hpart;
  size_t total;
};

Dims make_dims(const donof_problem* p);

// Storage of the split B for the half transform.  N > kDenseMaxN: lower-triangle tile
// storage, row tiles of 128 AO indices (T of them), the last one stored with its rows rounded
// up to a multiple of 64; tile (i, j), j <= i, holds rows of tile i and columns of tile j as
// chunks of 64 columns, each chunk [R_i rows][64] with the 16-byte pieces of row r at
// piece ^ (r % 8).  N <= kDenseMaxN (dense): every slice whole, [N][ld] with ld = N rounded up
// to 8 (a tensor-map row pitch of 16-byte multiples), read through a 3-D tensor map whose
// zero fill pads the 128-row tiles and 64-wide K steps; at these sizes the tiles' padding
// would cost more bytes than the dense copy of the upper triangle.
constexpr int kDenseMaxN = 256;
struct SymTiles {
  int T, Rlast;
  long long perP;  // elements per slice and plane
  int dense, ld;   // dense storage and its row pitch (elements)
};
__host__ __device__ inline int sym_R(const SymTiles& t, int i) { return i < t.T - 1 ? 128 : t.Rlast; }
__host__ __device__ inline long long sym_tile_off(const SymTiles& t, int i, int j) {
  return 16384LL * i * (i + 1) / 2 + (long long)sym_R(t, i) * 128 * j;
}
__host__ __device__ inline SymTiles sym_tiles(int N) {
  SymTiles t;
  t.T = (N + 127) / 128;
  const int last = N - 128 * (t.T - 1);
  t.Rlast = (last + 63) / 64 * 64;
  t.dense = N <= kDenseMaxN ? 1 : 0;
  t.ld = (N + 7) / 8 * 8;
  t.perP = t.dense ? (long long)N * t.ld
                   : sym_tile_off(t, t.T - 1, 0) + (long long)t.Rlast * (128LL * (t.T - 1) + t.Rlast);
  return t;
}

// ---------------------------------------------------------------------------
// Grouped launches (batch.cu): one launch runs a kernel for every instance of a batch.  A
// kernel body takes its block coordinates as a Blk (the native ones for a single instance);
// in a grouped launch instance i owns the blocks [start[i], start[i+1]) of the flat grid,
// laid out as its own grid of dims[3i .. 3i+2].
// ---------------------------------------------------------------------------
struct Blk {
  int x, y, z, gx, gy, gz;
};
__device__ __forceinline__ Blk native_blk() {
  return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
             (int)gridDim.x,  (int)gridDim.y,  (int)gridDim.z};
}
// One instance of a batch: its sizes, workspace carving and pointers.
struct InstRec {
  Dims d;
  Layout L;
  char* ws;
  const double *h, *B, *C, *gamma;
  const int32_t* pm;
  double *E, *lam, *dEdg, *dEdC;
  const double* Ebar;  // upstream gradient of the adjoint (1.0)
};
struct GroupLaunch {
  const InstRec* inst;
  const int* start;  // [ninst + 1]
  const int* dims;   // [3 ninst]
  int ninst;
};
// The instance of this block and its coordinates in that instance's grid.
__device__ __forceinline__ int group_locate(const GroupLaunch& g, Blk& b) {
  const int bid = (int)blockIdx.x;
  int lo = 0, hi = g.ninst - 1;
  while (lo < hi) {  // the last instance whose first block is at or before bid
    const int mid = (lo + hi + 1) >> 1;
    if (g.start[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  const int l = bid - g.start[lo];
  const int gx = g.dims[3 * lo], gy = g.dims[3 * lo + 1], gz = g.dims[3 * lo + 2];
  b.x = l % gx;
  b.y = (l / gx) % gy;
  b.z = l / (gx * gy);
  b.gx = gx;
  b.gy = gy;
  b.gz = gz;
  return lo;
}

// The K and J partials' entries (q, p0..p0+3) on and below the diagonal (p0 <= q, p0 a
// multiple of 4), row by row: rows 4k .. 4k+3 have k + 1 such quads each, so the rows before
// 4k hold 2k(k+1) of them.
__host__ __device__ inline int kpart_quads(int A) {
  const int kb = A / 4;
  return 2 * kb * (kb + 1) + (A % 4) * (kb + 1);
}

// Tiles of k_diag_w (mid.cu): a CTA per 32 slices and 64 columns.
constexpr int kDiagWTileSlices = 32, kDiagWTileCols = 64;

// The grouped launches of one batched build, in order (batch.cu builds their grids).
enum GroupKind {
  GK_ZERO, GK_OCC, GK_COEF, GK_SPLIT_C, GK_TC_HC, GK_SUM_HC, GK_GRAM_PART, GK_GRAM_FINAL,
  GK_HDIAG, GK_XEXP, GK_TC_HALF, GK_TC_B, GK_DIAGW, GK_KPART, GK_JKEY, GK_YQUANT, GK_TC_G,
  GK_REDUCEG, GK_EROWS, GK_EFINAL, GK_SPLIT_L, GK_TC_LAM, GK_SUM_L, GK_BWD, GK_COUNT
};
// Host launchers of the grouped kernels (blocks: the flat grid; threads, smem per block).
cudaError_t launch_fp64_group(int kind, const GroupLaunch& g, int blocks, int threads,
                              size_t smem, cudaStream_t s);
cudaError_t launch_mid_group(int kind, const GroupLaunch& g, int blocks, dim3 threads,
                             cudaStream_t s);
cudaError_t launch_tc_small_group(int kind, const GroupLaunch& g, int blocks, int threads,
                                  cudaStream_t s);
// Grouped tensor-core contractions (kind GK_TC_*; tc.cu): their argument and tensor-map
// records are opaque here, byte records of tc_args_bytes() and tc_maps_bytes() each (maps
// 64-byte aligned).  Setup fills instance records on the host and counts its work units;
// finish writes the kernel-wide settings into all records and returns the launch's shared
// memory and its numeric mode (cat: the planes of B concatenated, for narrow tiles); the
// launch reads the records from device memory.
bool tc_group_setup(int kind, const Dims& d, char* ws, const Layout& L, void* a_rec,
                    void* m_rec, int& units);
size_t tc_group_finish(int kind, void* a_recs, int ninst, int* status, int* abort_flag,
                       int& cat);
cudaError_t launch_tc_group(int kind, const void* args_dev, const void* maps_dev,
                            const int* ustart, int ninst, int units, size_t smem, int cat,
                            cudaStream_t s);
size_t tc_args_bytes();
size_t tc_maps_bytes();

// Tracing (api.cu): no-ops unless donof_profile_enable(1) was called.
void prof_begin(int phase, cudaStream_t s);
void prof_end(int phase, cudaStream_t s);
void count_launch(int n);
Layout make_layout(const Dims& d);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ inline void set_status(DevHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// Integer + fraction split of the tensor-core operands.  A vector x of K elements is
// 2^e (h + f) with y = x / 2^e, h = rint(y) rounded to fp16 (exact up to 2048, even
// integers up to 4096) and f = fp16(y - h).  e is the smallest exponent with
// ||y||_2 < T = 2^12 - sqrt(K)/2 - 2: then at most three elements exceed 2048, so
// |h - y| <= 1/2 elementwise except there (<= 3/2), ||h - y||_2 <= sqrt(K)/2 + 2 and
// ||h||_2 < 2^12.  For two such vectors every partial sum of h_a h_b is an integer below
// 2^24 in magnitude (Cauchy-Schwarz), so the integer products accumulate exactly in fp32.
// `nrm` must bound ||x||_2.
// 1/T rounded up (relative 2^-50), so that nrm * intfrac_inv_target(K) >= nrm / T after
// rounding: the exponent below never comes out too small.  Computed once per launch (the
// FP64 square root and division are slow on this GPU).
__host__ __device__ inline double intfrac_inv_target(double K) {
  double T = 4096.0 - 0.5 * sqrt(K) - 2.0;
  if (T < 1024.0) T = 1024.0;  // K above 3.7e7: exactness no longer guaranteed, values still
                               // represented to within the fp16 fraction
  return (1.0 / T) * (1.0 + 0x1p-50);
}
__host__ __device__ inline int intfrac_exponent_inv(double nrm, double invT) {
  if (!(nrm > 0.0)) return 0;
  int e;
  frexp(nrm * invT, &e);  // nrm / T <= nrm * invT < 2^e
  return e;
}
__host__ __device__ inline int intfrac_exponent(double nrm, double K) {
  return intfrac_exponent_inv(nrm, intfrac_inv_target(K));
}
// Exponent of a row from its squared norm, without the FP64 square root: the smallest e
// with sqrt(nrm2) / T < 2^e, from x = nrm2 * invT2 (invT2 >= 1/T^2 after rounding):
// x < 2^e2 gives sqrt(nrm2) / T <= sqrt(x) < 2^(e2/2) <= 2^ceil(e2/2).
__host__ __device__ inline double intfrac_inv_target_sq(double K) {
  const double i = intfrac_inv_target(K);
  return (i * i) * (1.0 + 0x1p-50);
}
__host__ __device__ inline int intfrac_exponent_sq(double nrm2, double invT2) {
  if (!(nrm2 > 0.0)) return 0;
  int e2;
  frexp(nrm2 * invT2, &e2);
  return e2 >= 0 ? (e2 + 1) / 2 : -((-e2) / 2);  // ceil(e2 / 2)
}
// 2^e as a double, exact for -1022 <= e <= 1023 (the exponents here are far inside)
__device__ inline double pow2d(int e) {
  e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  return __longlong_as_double((long long)(e + 1023) << 52);
}
// The integer + fraction split (and its residual) of y = v 2^k for a double v, formed in
// fp32 (this GPU's FP64 pipe is narrow): v as the two-float vh + vl (vh = fl32(v), vl =
// fl32(v - vh), within 2^-48 |v|); both scaled by 2^k exactly; h = fp16(rint(yh)) (even
// above 2048), dh = yh - h (exact: |yh| < 2^12), f = fp16(dh + yl), r = fp16((dh - f) + yl).  The same h and f as the
// double split up to rounding ties (h may then be the other neighbour of y, |y - h| a few
// units of 2^-24 above 1/2), r to about 2^-36 of the unit of h.  Outside the normal range of
// a float scale (|k| > 120) the double arithmetic is used.
__device__ inline void intfrac_split_v(double v, int k, __half& h, __half& f, __half& r) {
  if (k < -120 || k > 120) {
    const double y = v * __longlong_as_double((long long)(k + 1023) << 52);
    const float hf = (float)rint(y);
    h = __float2half_rn(hf);
    f = __float2half_rn((float)(y - (double)__half2float(h)));
    r = __double2half((y - (double)__half2float(h)) - (double)__half2float(f));
    return;
  }
  const float vh = __double2float_rn(v);
  const float vl = __double2float_rn(v - (double)vh);
  const float sc = __int_as_float((k + 127) << 23);
  const float yh = vh * sc, yl = vl * sc;
  h = __float2half_rn(rintf(yh));
  const float dh = yh - __half2float(h);  // h as stored (even above 2048): exact
  f = __float2half_rn(dh + yl);
  r = __float2half_rn((dh - __half2float(f)) + yl);
}
__device__ inline void intfrac_split(double y, __half& h, __half& f) {
  const float hf = (float)rint(y);  // exact: |y| < 4096
  h = __float2half_rn(hf);
  f = __float2half_rn((float)(y - (double)__half2float(h)));
}
__device__ inline void intfrac_split(float y, __half& h, __half& f) {
  h = __float2half_rn(rintf(y));
  f = __float2half_rn(y - __half2float(h));  // exact difference: |y| < 4096
}

// ---------------------------------------------------------------------------
// Kernel launchers (host side), implemented in fp64.cu and tc.cu.
// All return a cudaError_t of the launch.
// ---------------------------------------------------------------------------

// C[b](m, n) = alpha * sum_{kb, k} A(m, kb, k) B(kb, k, n) + beta * C[b](m, n)
// with A(m, kb, k) = A[b*sAb + m*sAm + kb*sAkb + k*sAk] and
//      B(kb, k, n) = B[b*sBb + kb*sBkb + k*sBk + n*sBn];
// Ktot > 0 limits the flattened contraction index kb*K + k to [0, Ktot) (used to split one
// long contraction into KB chunks of K that ksplit CTAs share).
// Output tile width of k_dgemm: 32 where it pads the width less than 64 does.
inline int dgemm_tile_n(int N) { return (N + 31) / 32 * 32 < (N + 63) / 64 * 64 ? 32 : 64; }
// ksplit > 1 (batch 1 only): each CTA stores its partial product alpha * A B over its share
// of the kb range in part[ks][M][N], and a second kernel adds the ksplit partials to C in
// order of ks (C += sum, so beta must be 1): the result does not depend on scheduling.
struct DgemmArgs {
  int M, N, K, KB, batch, ksplit, Ktot;
  int lower;  // 1: only output tiles that reach the lower triangle (m >= n); ksplit == 1
  const double* A; long long sAb, sAm, sAk, sAkb;
  const double* B; long long sBb, sBk, sBn, sBkb;
  double* C; long long sCb, sCm, sCn;
  double alpha, beta;
  double* part;  // ksplit x M x N scratch when ksplit > 1
};
cudaError_t launch_dgemm(const DgemmArgs& a, cudaStream_t s);
// The split count split_k_args uses for an M x N output with contraction length K.
int splitk_count(int M, int N, int K);
// Symmetric FP64 eigensolver (eigh.cu): A (N x N, row-major, symmetric; not modified) =
// V diag(w) V^T with w ascending and V row-major (column j = eigenvector j).  V may share
// A's storage.  Workspace: eigh_workspace_bytes(N), 256-byte aligned, its first bytes the
// solver's device header.
constexpr int kEighMaxN = 4096;
size_t eigh_workspace_bytes(int N);
int eigh_run(int N, const double* A, double* V, double* w, char* ws, cudaStream_t s);
int g_splits_fp64(int N, int A, int np);
// C(m, n) += sum_k A(m, k) B(k, n) with the contraction cut into 64-wide (or 16-wide) chunks
// shared by enough CTAs to fill the GPU; `part` holds splitk_count(M, N, K) x M x N doubles
// (C must be initialised).
DgemmArgs split_k_args(int M, int N, int K, const double* A, long long sAm, long long sAk,
                       const double* B, long long sBk, long long sBn, double* C, long long sCm,
                       long long sCn, double* part);

cudaError_t launch_occupations(const Dims& d, const double* gamma, const int32_t* pair_map,
                               char* ws, const Layout& L, cudaStream_t s);
cudaError_t launch_coefficients(const Dims& d, const int32_t* pair_map, char* ws, const Layout& L,
                                cudaStream_t s);
cudaError_t launch_unpack_B(const Dims& d, const double* Bp, int p0, int np, double* out,
                            cudaStream_t s);
// H_pp = C_p^T h C_p and G = n o (h C_act) (one_electron_G), or G = 0 (the partial sums of
// one shard of a sharded build carry only the two-electron part).
cudaError_t launch_hdiag_ginit(const Dims& d, const double* C, char* ws, const Layout& L,
                               bool one_electron_G, cudaStream_t s);
// y += x over n doubles.
cudaError_t launch_add(double* y, const double* x, long long n, cudaStream_t s);
cudaError_t launch_jk_accumulate_f64(const Dims& d, const double* b, int np, int ld, char* ws,
                                     const Layout& L, cudaStream_t s);

cudaError_t launch_build_Y_f64(const Dims& d, const double* b, double* Y, int np, char* ws,
                               const Layout& L, cudaStream_t s);

// Mixed path between the b and G contractions (mid.cu): J, K and the Y operand split.
cudaError_t launch_mid_mixed(const Dims& d, int np, int splits, char* ws, const Layout& L,
                             cudaStream_t s);

cudaError_t launch_energy(const Dims& d, const int32_t* pair_map, char* ws, const Layout& L,
                          double* E_out, double* dEdg_out, cudaStream_t s);
cudaError_t launch_backward(const Dims& d, const double* Ebar, const char* ws, const Layout& L,
                            double* dE_dC, double* dE_dgamma, cudaStream_t s);

// mixed path
cudaError_t launch_prepare_split_B(const Dims& d, const double* B, char* ws, const Layout& L,
                                   cudaStream_t s);
// The splits of C_act^T (for b and for h C_act), of diag(2^s) C_act (half transform) and of
// h (for h C_act), in two launches.
// with_half_transform = false leaves out the operand of the half transform (its exponents
// come from the prepared B), for a build that runs no contraction over B.
cudaError_t launch_split_C(const Dims& d, const double* C, const double* h, char* ws,
                           const Layout& L, bool with_half_transform, cudaStream_t s);
// hC = h C_act on the tensor cores from the planes written by launch_split_C (mixed path).
int run_hc_tc(const Dims& d, char* ws, const Layout& L, cudaStream_t s);
cudaError_t launch_reduce_G(const Dims& d, char* ws, const Layout& L, cudaStream_t s);
cudaError_t launch_gram_bound(const Dims& d, const double* C, char* ws, const Layout& L,
                              cudaStream_t s);
// The three tensor-core contractions of one block of np auxiliary slices starting at p0.
int run_tc_block(const Dims& d, int p0, int np, char* ws, const Layout& L, cudaStream_t s);
// lambda = C^T G on the tensor cores with residual-extended operands (mixed path).
int run_lambda_tc(const Dims& d, const double* C, char* ws, const Layout& L, double* lam,
                  cudaStream_t s);

}  // namespace donof
