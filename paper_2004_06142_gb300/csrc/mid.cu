// Mixed path, between the b contraction and the G contraction: from the MO three-index
// slices b^P (fp32, [P][q][p], pitch Ap) to J, K (Eq. JKpq in density-fitted form) and to
// the integer + fraction operand of the G contraction,
//   Y^P_qp = Bcoef_qp b^P_qp + delta_qp w^P_p,   w^P_p = sum_r Acoef_pr d^P_r,  d^P_r = b^P_rr,
// (the J and K coefficient matrices of E applied slice by slice, Eqs. Vee-s, Vee-d), without
// materialising Y in fp32:
//   k_diag_w   w^P per slice from d^P (written by the b contraction; fp32, W = D Acoef in tiles);
//   k_kpart    per G split sp: Ksp_qp = sum_{P in sp} (b^P_qp)^2 and Jsp_qp = sum d^P_q d^P_p
//              (fp32 groups of 16 slices, double across groups), b read once;
//   k_jk_eY    K += sum_sp Ksp, J += sum_sp Jsp (double, fixed order), and the exponent of
//              row p of Y over split sp from its exact squared norm
//                sum_q Bcoef_qp^2 Ksp_qp + 2 Bcoef_pp sum_P d^P_p w^P_p + sum_P (w^P_p)^2;
//   k_y_quant  Y computed on the fly and written as integer + fraction planes, b read again.
#include "common.cuh"

namespace donof {
namespace {

__device__ __forceinline__ float pow2f_m(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((e + 127) << 23);
}


// w^P = Acoef d^P for every slice, from the diagonals d^P of b^P that the b contraction wrote
// into D, as the product W = D Acoef (Acoef symmetric) in tiles: a CTA of 256 threads per 32
// slices and 64 columns p, the d and Acoef tiles of 64 r at a time in shared memory; thread
// (p, g) forms w_p of slices 8g .. 8g+7, the products added in order of r.
constexpr int kDwS = kDiagWTileSlices, kDwP = kDiagWTileCols, kDwR = 64;
__device__ __forceinline__ void k_diag_w_body(const Blk& B_, const float* __restrict__ D, int np,
                                              int A, int Ap, const float* __restrict__ AcF,
                                              float* W) {
  __shared__ float dT[kDwS][kDwR + 1];
  __shared__ float At[kDwR][kDwP];
  const int P0 = B_.x * kDwS, p0 = B_.y * kDwP;
  const int tid = threadIdx.x, pl = tid % kDwP, sg = tid / kDwP;
  float w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = 0.f;
  for (int r0 = 0; r0 < A; r0 += kDwR) {
    const int nr = min(kDwR, A - r0);
    for (int i = tid; i < kDwS * kDwR; i += blockDim.x) {
      const int sl = i / kDwR, r = i % kDwR;
      dT[sl][r] = (P0 + sl < np && r < nr) ? D[(size_t)(P0 + sl) * A + r0 + r] : 0.f;
    }
    for (int i = tid; i < kDwR * kDwP; i += blockDim.x) {
      const int r = i / kDwP, c = i % kDwP;
      At[r][c] = (r < nr && p0 + c < A) ? AcF[(size_t)(r0 + r) * Ap + p0 + c] : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const float a = At[r][pl];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = fmaf(a, dT[sg * 8 + k][r], w[k]);
    }
    __syncthreads();
  }
  const int p = p0 + pl;
  if (p < A) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int P = P0 + sg * 8 + k;
      if (P < np) W[(size_t)P * A + p] = w[k];
    }
  }
}
__global__ void __launch_bounds__(256) k_diag_w(const float* __restrict__ D, int np, int A,
                                                int Ap, const float* __restrict__ AcF,
                                                float* W) {
  k_diag_w_body(native_blk(), D, np, A, Ap, AcF, W);
}

// Per split: K and J partials of four consecutive entries (q, p0..p0+3) per thread, a thread
// per quad with p0 <= q (K and J are symmetric: every entry with p <= q is formed, read by
// k_jk_eY for its mirror too, so that b is read on and below the diagonal only).
__device__ __forceinline__ void kpart_quad(int i, int& q, int& p0) {
  int k = (int)((sqrtf(1.f + 2.f * (float)i) - 1.f) * 0.5f);
  while (2 * (k + 1) * (k + 2) <= i) ++k;
  while (2 * k * (k + 1) > i) --k;
  const int r = i - 2 * k * (k + 1);
  q = 4 * k + r / (k + 1);
  p0 = 4 * (r % (k + 1));
}
__device__ __forceinline__ void k_kpart_body(const Blk& B_, const float* __restrict__ b,
                                               const float* __restrict__ D, int np, int A,
                                               int Ap, int splits, double* Ksp, double* Jsp) {
  const int i4 = B_.x * blockDim.x + threadIdx.x;  // a quad on or below the diagonal
  const int sp = B_.y;
  if (i4 >= kpart_quads(A)) return;
  int q, p0;
  kpart_quad(i4, q, p0);
  const int P0 = (int)((long long)np * sp / splits), P1 = (int)((long long)np * (sp + 1) / splits);
  double sk[4] = {0.0, 0.0, 0.0, 0.0}, sj[4] = {0.0, 0.0, 0.0, 0.0};
  const float4* b4 = (const float4*)b;
  const size_t slice4 = (size_t)Ap * Ap / 4;
  const size_t e4 = (size_t)q * (Ap / 4) + p0 / 4;
  for (int G0 = P0; G0 < P1; G0 += 16) {
    const int G1 = min(P1, G0 + 16);
    float fk[4] = {0.f, 0.f, 0.f, 0.f}, fj[4] = {0.f, 0.f, 0.f, 0.f};
    for (int Pb = G0; Pb < G1; Pb += 8) {
      // eight slices' loads in flight, then the products added in order of P
      float4 v[8];
      float dq[8], dp[8][4];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int P = Pb + u;
        const bool in = P < G1;
        const float* dP = D + (size_t)(in ? P : Pb) * A;
        v[u] = in ? b4[(size_t)P * slice4 + e4] : make_float4(0.f, 0.f, 0.f, 0.f);
        dq[u] = in ? dP[q] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) dp[u][j] = (in && p0 + j < A) ? dP[p0 + j] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (Pb + u < G1) {
          fk[0] = fmaf(v[u].x, v[u].x, fk[0]);
          fk[1] = fmaf(v[u].y, v[u].y, fk[1]);
          fk[2] = fmaf(v[u].z, v[u].z, fk[2]);
          fk[3] = fmaf(v[u].w, v[u].w, fk[3]);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (p0 + j < A) fj[j] = fmaf(dq[u], dp[u][j], fj[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sk[j] += fk[j];
      sj[j] += fj[j];
    }
  }
  const size_t o = ((size_t)sp * A + q) * A + p0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (p0 + j < A) {
      Ksp[o + j] = sk[j];
      Jsp[o + j] = sj[j];
    }
}
__global__ void __launch_bounds__(256) k_kpart(const float* __restrict__ b,
                                               const float* __restrict__ D, int np, int A,
                                               int Ap, int splits, double* Ksp, double* Jsp) {
  k_kpart_body(native_blk(), b, D, np, A, Ap, splits, Ksp, Jsp);
}

// K += sum_sp Ksp, J += sum_sp Jsp (entries of blocks x), then the Y row exponents (blocks y).
__device__ __forceinline__ void k_jk_eY_body(const Blk& B_, const double* __restrict__ Ksp,
                                               const double* __restrict__ Jsp,
                                               const float* __restrict__ D,
                                               const float* __restrict__ W,
                                               const float* __restrict__ BcF, int np, int A,
                                               int Ap, int splits, double* K, double* J,
                                               int* eY) {
  const int AA = A * A;
  // blocks x < n0: the K, J sums (a thread per entry); the others: the exponents
  const int n0 = (AA + blockDim.x - 1) / blockDim.x;
  if (B_.x < n0) {
    {
      const int i = B_.x * blockDim.x + threadIdx.x;
      if (i >= AA) return;
      const int qi = i / A, pi = i % A;
      const int src = pi <= qi ? i : pi * A + qi;  // the partials hold p <= q
      double k = 0.0, j = 0.0;
      int sp = 0;
      for (; sp + 8 <= splits; sp += 8) {  // eight splits in flight, summed in order
        double kv[8], jv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          kv[u] = Ksp[(size_t)(sp + u) * AA + src];
          jv[u] = Jsp[(size_t)(sp + u) * AA + src];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          k += kv[u];
          j += jv[u];
        }
      }
      for (; sp < splits; ++sp) {
        k += Ksp[(size_t)sp * AA + src];
        j += Jsp[(size_t)sp * AA + src];
      }
      K[i] += k;
      J[i] += j;
    }
    return;
  }
  // one warp per (split, row p), rows p >= A get exponent 0
  const int lane = threadIdx.x % 32;
  const int nrow = splits * Ap;
  for (int t = ((B_.x - n0) * blockDim.x + threadIdx.x) / 32; t < nrow;
       t += (B_.gx - n0) * blockDim.x / 32) {
    const int sp = t / Ap, p = t % Ap;
    // the squared norm in fp32 (this GPU's FP64 pipe is narrow): ss, and sa the sum of the
    // terms' magnitudes; fewer than 64 roundings of 2^-24 each (conversions included) keep
    // ss within 2^-17 sa of the exact sum, so ss + 2^-16 sa bounds it from above
    float ss = 0.f, sa = 0.f;
    if (p < A) {
      const double* Ks = Ksp + (size_t)sp * AA;
      for (int q = lane; q < A; q += 32) {
        const float bc = BcF[(size_t)q * Ap + p];
        const float t2 = bc * bc * (float)Ks[q >= p ? (size_t)q * A + p : (size_t)p * A + q];
        ss += t2;
        sa += t2;
      }
      const int P0 = (int)((long long)np * sp / splits);
      const int P1 = (int)((long long)np * (sp + 1) / splits);
      const float bpp = BcF[(size_t)p * Ap + p];
      for (int P = P0 + lane; P < P1; P += 32) {
        const float d = D[(size_t)P * A + p], w = W[(size_t)P * A + p];
        const float c = 2.f * bpp * d * w, w2 = w * w;
        ss += c + w2;
        sa += fabsf(c) + w2;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    const double bound = (double)ss + 0x1p-16 * (double)sa;
    // row length of the G contraction over this split: (slices in it) x Ap
    const double Kc = (double)(np * (sp + 1LL) / splits - np * (long long)sp / splits) * Ap;
    if (lane == 0) eY[t] = intfrac_exponent(sqrt(fmax(bound, 0.0)) * (1.0 + 1e-6), Kc);
  }
}
__global__ void __launch_bounds__(256) k_jk_eY(const double* __restrict__ Ksp,
                                               const double* __restrict__ Jsp,
                                               const float* __restrict__ D,
                                               const float* __restrict__ W,
                                               const float* __restrict__ BcF, int np, int A,
                                               int Ap, int splits, double* K, double* J,
                                               int* eY) {
  k_jk_eY_body(native_blk(), Ksp, Jsp, D, W, BcF, np, A, Ap, splits, K, J, eY);
}

// Y^P_rc = Bcoef_rc b^P_rc + delta_rc w^P_r -> integer + fraction planes with row exponent
// eY[spOf[P]][r]: a CTA per slice at a time, thread (c4, y) handles four consecutive entries
// of rows r = y, y + 8, ... (blockDim = (Ap / 4, 8)).
__device__ __forceinline__ void k_y_quant_body(const Blk& B_, const float* __restrict__ b, const float* __restrict__ W,
                          const float* __restrict__ BcF, int np, int A, int Ap,
                          const int* __restrict__ spOf, const int* __restrict__ eY,
                          __half* __restrict__ H, __half* __restrict__ F, DevHeader* hdr) {
  if (B_.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    hdr->e3 = 0;  // G partials are in true units
  const int r4 = Ap / 4, c4 = threadIdx.x, c0 = 4 * c4;
  const float4* Bc4 = (const float4*)BcF;
  for (int P = B_.x; P < np; P += B_.gx) {
    const float4* b4 = (const float4*)b + (size_t)P * Ap * r4;
    const int* eYs = eY + (size_t)spOf[P] * Ap;
    constexpr int kRows = 4;  // rows of a thread whose loads are in flight together
    for (int r0 = threadIdx.y; r0 < Ap; r0 += kRows * blockDim.y) {
      float4 v[kRows], bc[kRows];
      int ey[kRows];
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int r = r0 + k * blockDim.y;
        const bool in = r < Ap;
        v[k] = in ? b4[(size_t)r * r4 + c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        bc[k] = in ? Bc4[(size_t)r * r4 + c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        ey[k] = in ? eYs[r] : 0;
      }
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int r = r0 + k * blockDim.y;
        if (r >= Ap) break;
        const float sc = pow2f_m(-ey[k]);
        float y[4] = {bc[k].x * v[k].x, bc[k].y * v[k].y, bc[k].z * v[k].z, bc[k].w * v[k].w};
        if (r < A && r >= c0 && r < c0 + 4) y[r - c0] += W[(size_t)P * A + r];
        __align__(8) __half h[4], fr[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) intfrac_split(y[j] * sc, h[j], fr[j]);
        const size_t o = ((size_t)P * Ap + r) * Ap + c0;
        *(uint2*)(H + o) = *(uint2*)h;
        *(uint2*)(F + o) = *(uint2*)fr;
      }
    }
  }
}
__global__ void k_y_quant(const float* __restrict__ b, const float* __restrict__ W,
                          const float* __restrict__ BcF, int np, int A, int Ap,
                          const int* __restrict__ spOf, const int* __restrict__ eY,
                          __half* __restrict__ H, __half* __restrict__ F, DevHeader* hdr) {
  k_y_quant_body(native_blk(), b, W, BcF, np, A, Ap, spOf, eY, H, F, hdr);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Grouped launches (every instance of a batch, one block of np = naux slices each, the G
// contraction's split count min(splits, np)).
__device__ __forceinline__ int group_splits(const Dims& d) { return d.splits < d.Q ? d.splits : d.Q; }
__global__ void __launch_bounds__(256) k_diag_w_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  const Dims& d = I.d;
  char* ws = I.ws;
  k_diag_w_body(b, (const float*)(ws + I.L.D), d.Q, d.A, d.Ap, (const float*)(ws + I.L.AcF),
                (float*)(ws + I.L.W));
}
__global__ void __launch_bounds__(256) k_kpart_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  const Dims& d = I.d;
  char* ws = I.ws;
  k_kpart_body(b, (const float*)(ws + I.L.b32), (const float*)(ws + I.L.D), d.Q, d.A, d.Ap,
               group_splits(d), (double*)(ws + I.L.Ksp), (double*)(ws + I.L.Jsp));
}
__global__ void __launch_bounds__(256) k_jk_eY_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  const Dims& d = I.d;
  char* ws = I.ws;
  k_jk_eY_body(b, (const double*)(ws + I.L.Ksp), (const double*)(ws + I.L.Jsp),
               (const float*)(ws + I.L.D), (const float*)(ws + I.L.W),
               (const float*)(ws + I.L.BcF), d.Q, d.A, d.Ap, group_splits(d),
               (double*)(ws + I.L.K), (double*)(ws + I.L.J), (int*)(ws + I.L.eY));
}
// blockDim.x is that of the widest instance (Ap / 4); the threads past this instance's
// Ap / 4 columns have nothing to do (the body has no block-wide barrier)
__global__ void k_y_quant_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  const Dims& d = I.d;
  if ((int)threadIdx.x >= d.Ap / 4) return;
  char* ws = I.ws;
  k_y_quant_body(b, (const float*)(ws + I.L.b32), (const float*)(ws + I.L.W),
                 (const float*)(ws + I.L.BcF), d.Q, d.A, d.Ap, (const int*)(ws + I.L.spOf),
                 (const int*)(ws + I.L.eY), (__half*)(ws + I.L.Yhi), (__half*)(ws + I.L.Ylo),
                 (DevHeader*)(ws + I.L.header));
}

}  // namespace

cudaError_t launch_mid_group(int kind, const GroupLaunch& g, int blocks, dim3 threads,
                             cudaStream_t s) {
  switch (kind) {
    case GK_DIAGW: k_diag_w_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_KPART: k_kpart_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_JKEY: k_jk_eY_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_YQUANT: k_y_quant_group<<<blocks, threads, 0, s>>>(g); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_mid_mixed(const Dims& d, int np, int splits, char* ws, const Layout& L,
                             cudaStream_t s) {
  const int A = d.A, Ap = d.Ap;
  const float* b = (const float*)(ws + L.b32);
  float* D = (float*)(ws + L.D);
  float* W = (float*)(ws + L.W);
  const float* AcF = (const float*)(ws + L.AcF);
  const float* BcF = (const float*)(ws + L.BcF);
  k_diag_w<<<dim3((np + kDwS - 1) / kDwS, (A + kDwP - 1) / kDwP), 256, 0, s>>>(D, np, A, Ap, AcF,
                                                                           W);
  k_kpart<<<dim3((kpart_quads(A) + 255) / 256, splits), 256, 0, s>>>(b, D, np, A, Ap, splits,
                                                         (double*)(ws + L.Ksp),
                                                         (double*)(ws + L.Jsp));
  const int ncta_e = (splits * Ap + 7) / 8;  // a warp per (split, row) of the exponents
  k_jk_eY<<<(A * A + 255) / 256 + ncta_e, 256, 0, s>>>((const double*)(ws + L.Ksp),
                                             (const double*)(ws + L.Jsp), D, W, BcF, np, A, Ap,
                                             splits, (double*)(ws + L.K), (double*)(ws + L.J),
                                             (int*)(ws + L.eY));
  k_y_quant<<<np < sm_count() * 8 ? np : sm_count() * 8, dim3(Ap / 4, 8), 0, s>>>(
      b, W, BcF, np, A, Ap, (const int*)(ws + L.spOf), (const int*)(ws + L.eY),
      (__half*)(ws + L.Yhi), (__half*)(ws + L.Ylo), (DevHeader*)(ws + L.header));
  count_launch(4);
  return cudaGetLastError();
}


}  // namespace donof
