// mpnn.cu -- the learned warm start.
//
// The paper starts every SCC's power series from P_0 = W (Sec. 4.3.2).  A
// guess R0 close to the solution shortens the series: continuing from the
// residual r = W + cA^T(R0/outdeg) - R0 needs log(||r||/tau)/log(1/c)
// sweeps instead of log(||W||/tau)/log(1/c).  The solution of an SCC is
// R_C = W_C + M_C W_C with M_C = (I - c A_C^T)^-1 - I >= 0, so R_i - W_i is
// about b_i mean_C(W), b_i being row i's amplification.  A small network
// over the SCC's internal in-edges guesses b_i from the structure alone
// (per SCC vertex i of component C: internal in-degree d_i, internal
// out-degree o_i, external in-degree e_i):
//   x_i  = [log1p(d_i), log1p(outdeg_i), log|C|, o_i/outdeg_i, log1p(e_i),
//           log1p(outdeg_i - o_i), 1, 0]
//   h_i  = relu(A1 x_i + B1 mean_{j->i} x_j + b1)           (64)
//   g_i  = relu(A2 h_i + B2 mean_{j->i} h_j + b2)           (64)
//   yhat = v . g_i + b3
// trained on y_i = log(max((R_i - W_i)/mean_C(W), 1e-6)) of solved graphs
// with the mean squared error.  The guess is
//   R0_i = W_i + exp(clamp(yhat_i, -14, 9)) mean_C(W),
// formed by the solver from the level's W when the level is reached, so the
// network runs once per partition and model (its inputs are structural).
// Weights are kept in float32 for the optimiser (Adam) and rounded to
// bfloat16 for the forward pass; sums are float32.  The forward pass is a
// gather of neighbour features (memory bound) followed by a 64 x 128
// matrix-vector product per vertex on the FP32 pipes.
#include <math.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "common.cuh"
#include "mpnn.cuh"

namespace prgb {

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// float32 -> nearest bfloat16, ties to even (add half an ulp of bfloat16 and
// the parity bit, keep the top 16 bits)
__host__ __device__ __forceinline__ uint16_t f2bf(float f) {
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  memcpy(&u, &f, 4);
#endif
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

__global__ void mp_to_bf16_k(int count, const float* __restrict__ w, uint16_t* __restrict__ w16) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) w16[i] = f2bf(w[i]);
}

__device__ __forceinline__ bool mp_is_scc(const int32_t* p_comp, const uint8_t* c_type, int p) {
  return c_type[p_comp[p]] == PR_TYPE_SCC;
}

struct MpLayout {
  int32_t r0, r1;
  const int32_t* int_ptr;
  const int32_t* int_idx;
  const int32_t* ext_ptr;
  const int32_t* p_outdeg;
  const int32_t* p_comp;
  const int32_t* c_off;
  const uint8_t* c_type;
};

static MpLayout mp_layout(const pr_partition_s* P, int32_t r0, int32_t r1) {
  MpLayout L;
  L.r0 = r0;
  L.r1 = r1;
  L.int_ptr = P->int_ptr;
  L.int_idx = P->int_idx;
  L.ext_ptr = P->ext_ptr;
  L.p_outdeg = P->p_outdeg;
  L.p_comp = P->p_comp;
  L.c_off = P->c_off;
  L.c_type = P->c_type;
  return L;
}

// row index of an internal in-neighbour (it lies in the range by
// construction: an SCC is inside one level)
__device__ __forceinline__ int mp_row(const MpLayout& L, int q, Ctl* ctl) {
  if (q < L.r0 || q >= L.r1) {
    if (ctl) set_err(ctl, PR_EINTERNAL, 401);
    return -1;
  }
  return q - L.r0;
}

// ---- features ---------------------------------------------------------------
// internal out-degree of the SCC rows of the range: a warp per row adds one
// to the source of each internal in-edge (dout zeroed by the caller)
__global__ void mp_dout_k(MpLayout L, int32_t* __restrict__ dout, Ctl* ctl) {
  const int rows = L.r1 - L.r0;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < rows; i += nw) {
    const int p = L.r0 + (int)i;
    if (!mp_is_scc(L.p_comp, L.c_type, p)) continue;  // warp-uniform
    for (int e = L.int_ptr[p] + lane; e < L.int_ptr[p + 1]; e += 32) {
      const int j = mp_row(L, L.int_idx[e], ctl);
      if (j >= 0) atomicAdd(&dout[j], 1);
    }
  }
}

__global__ void mp_feat_k(MpLayout L, const int32_t* __restrict__ dout, float* __restrict__ X) {
  const int rows = L.r1 - L.r0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const int p = L.r0 + i;
    float x[kMpF0] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (mp_is_scc(L.p_comp, L.c_type, p)) {
      const int c = L.p_comp[p];
      const int od = L.p_outdeg[p], o = dout[i];
      x[0] = log1pf((float)(L.int_ptr[p + 1] - L.int_ptr[p]));
      x[1] = log1pf((float)od);
      x[2] = logf((float)(L.c_off[c + 1] - L.c_off[c]));
      x[3] = (float)o / (float)max(od, 1);
      x[4] = log1pf((float)(L.ext_ptr[p + 1] - L.ext_ptr[p]));
      x[5] = log1pf((float)(od - o));
      x[6] = 1.0f;
    }
    float4* out = reinterpret_cast<float4*>(X + (size_t)i * kMpF0);
    out[0] = make_float4(x[0], x[1], x[2], x[3]);
    out[1] = make_float4(x[4], x[5], x[6], x[7]);
  }
}

// ---- layer 1: thread per row ------------------------------------------------
__global__ void __launch_bounds__(kBlock) mp_l1_k(MpLayout L, const float* __restrict__ X,
                                                  const uint16_t* __restrict__ w16, float* __restrict__ H1,
                                                  float* __restrict__ M1, Ctl* ctl) {
  __shared__ float A1[kMpH * kMpF0], B1[kMpH * kMpF0], b1[kMpH];
  for (int t = threadIdx.x; t < kMpH * kMpF0; t += blockDim.x) {
    A1[t] = bf2f(w16[kMpA1 + t]);
    B1[t] = bf2f(w16[kMpB1 + t]);
  }
  for (int t = threadIdx.x; t < kMpH; t += blockDim.x) b1[t] = bf2f(w16[kMpb1 + t]);
  __syncthreads();
  const int rows = L.r1 - L.r0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const int p = L.r0 + i;
    float* h = H1 + (size_t)i * kMpH;
    if (!mp_is_scc(L.p_comp, L.c_type, p)) {
      for (int o = 0; o < kMpH; o++) h[o] = 0.0f;
      if (M1)
        for (int k = 0; k < kMpF0; k++) M1[(size_t)i * kMpF0 + k] = 0.0f;
      continue;
    }
    float x[kMpF0], m[kMpF0];
    for (int k = 0; k < kMpF0; k++) {
      x[k] = X[(size_t)i * kMpF0 + k];
      m[k] = 0.0f;
    }
    const int e0 = L.int_ptr[p], e1 = L.int_ptr[p + 1];
    for (int e = e0; e < e1; e++) {
      const int j = mp_row(L, L.int_idx[e], ctl);
      if (j < 0) continue;
      for (int k = 0; k < kMpF0; k++) m[k] += X[(size_t)j * kMpF0 + k];
    }
    const float inv = e1 > e0 ? 1.0f / (float)(e1 - e0) : 0.0f;
    for (int k = 0; k < kMpF0; k++) m[k] *= inv;
    if (M1)
      for (int k = 0; k < kMpF0; k++) M1[(size_t)i * kMpF0 + k] = m[k];
    for (int o = 0; o < kMpH; o++) {
      float z = b1[o];
#pragma unroll
      for (int k = 0; k < kMpF0; k++) z += A1[o * kMpF0 + k] * x[k] + B1[o * kMpF0 + k] * m[k];
      h[o] = fmaxf(z, 0.0f);
    }
  }
}

// ---- layer 2 and the head: warp per row, two features per lane -------------
// Weights transposed in shared memory ([k][o]) so that the lanes' outputs
// o = 2 lane, 2 lane + 1 read consecutive words.
constexpr size_t kMpL2Smem = (size_t)(2 * kMpH * kMpH + 2 * kMpH + (kBlock / 32) * 2 * kMpH) * sizeof(float);

__global__ void __launch_bounds__(kBlock) mp_l2_k(MpLayout L, const float* __restrict__ H1,
                                                  const uint16_t* __restrict__ w16, float* __restrict__ yhat,
                                                  float* __restrict__ G, float* __restrict__ M2, Ctl* ctl) {
  extern __shared__ float sm[];
  float* A2t = sm;                    // [k][o]
  float* B2t = sm + kMpH * kMpH;      // [k][o]
  float* b2 = sm + 2 * kMpH * kMpH;
  float* v = b2 + kMpH;
  float* stage = v + kMpH;            // per warp: h (64) then m (64)
  for (int t = threadIdx.x; t < kMpH * kMpH; t += blockDim.x) {
    const int o = t / kMpH, k = t % kMpH;
    A2t[k * kMpH + o] = bf2f(w16[kMpA2 + t]);
    B2t[k * kMpH + o] = bf2f(w16[kMpB2 + t]);
  }
  for (int t = threadIdx.x; t < kMpH; t += blockDim.x) {
    b2[t] = bf2f(w16[kMpb2 + t]);
    v[t] = bf2f(w16[kMpv + t]);
  }
  __syncthreads();
  const float b3 = bf2f(w16[kMpb3]);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sh = stage + wib * 2 * kMpH;
  const int rows = L.r1 - L.r0;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < rows; i += nw) {
    const int p = L.r0 + (int)i;
    const bool scc = mp_is_scc(L.p_comp, L.c_type, p);
    float2 g2 = make_float2(0.0f, 0.0f), m2 = make_float2(0.0f, 0.0f);
    float y = 0.0f;
    if (scc) {
      const float2 h2 = *reinterpret_cast<const float2*>(H1 + (size_t)i * kMpH + 2 * lane);
      const int e0 = L.int_ptr[p], e1 = L.int_ptr[p + 1];
      for (int e = e0; e < e1; e++) {
        const int j = mp_row(L, L.int_idx[e], ctl);
        if (j < 0) continue;
        const float2 t = *reinterpret_cast<const float2*>(H1 + (size_t)j * kMpH + 2 * lane);
        m2.x += t.x;
        m2.y += t.y;
      }
      const float inv = e1 > e0 ? 1.0f / (float)(e1 - e0) : 0.0f;
      m2.x *= inv;
      m2.y *= inv;
      sh[2 * lane] = h2.x;
      sh[2 * lane + 1] = h2.y;
      sh[kMpH + 2 * lane] = m2.x;
      sh[kMpH + 2 * lane + 1] = m2.y;
      __syncwarp();
      float z0 = b2[2 * lane], z1 = b2[2 * lane + 1];
#pragma unroll 8
      for (int k = 0; k < kMpH; k++) {
        const float hk = sh[k], mk = sh[kMpH + k];
        const float2 a = *reinterpret_cast<const float2*>(A2t + k * kMpH + 2 * lane);
        const float2 b = *reinterpret_cast<const float2*>(B2t + k * kMpH + 2 * lane);
        z0 += a.x * hk + b.x * mk;
        z1 += a.y * hk + b.y * mk;
      }
      g2 = make_float2(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f));
      float part = v[2 * lane] * g2.x + v[2 * lane + 1] * g2.y;
      y = group_sumf<32>(part) + b3;
      __syncwarp();  // the stage is rewritten by the next row
    }
    if (G) *reinterpret_cast<float2*>(G + (size_t)i * kMpH + 2 * lane) = g2;
    if (M2) *reinterpret_cast<float2*>(M2 + (size_t)i * kMpH + 2 * lane) = m2;
    if (lane == 0 && yhat) yhat[i] = y;
  }
}

// ---- training: targets, loss and the backward pass ---------------------------
// R by position and the inflow-adjusted weights it implies (Eq. PR:levels)
__global__ void mp_rpos_k(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ R,
                          double* __restrict__ Rp) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    Rp[p] = R[perm[p]];
}

__global__ void mp_w_k(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ u,
                       const double* __restrict__ Rp, const int32_t* __restrict__ ext_ptr,
                       const int32_t* __restrict__ ext_idx, const double* __restrict__ p_inv, double c,
                       double* __restrict__ W) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = ext_ptr[p]; e < ext_ptr[p + 1]; e++) {
      const int q = ext_idx[e];
      acc += Rp[q] * p_inv[q];
    }
    W[p] = u[perm[p]] + c * acc;
  }
}

// mean_C(W) of every SCC (a warp per component, a fixed-order sum)
__global__ void mp_cmean_k(int32_t K, const int32_t* __restrict__ c_off, const uint8_t* __restrict__ c_type,
                           const double* __restrict__ W, double* __restrict__ cmean) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < K; c += nw) {
    if (c_type[c] != PR_TYPE_SCC) continue;  // warp-uniform
    const int o0 = c_off[c], o1 = c_off[c + 1];
    double s = 0.0;
    for (int p = o0 + lane; p < o1; p += 32) s += W[p];
    s = group_sum<32>(s);
    if (lane == 0) cmean[c] = s / (double)(o1 - o0);
  }
}

// r_i = yhat_i - y_i on the rows of the SCCs with mean_C(W) > 0 (0
// elsewhere), y_i = log(max((R_i - W_i) / mean_C(W), 1e-6)); its squared
// sum and the row count
__global__ void mp_resid_k(int32_t n, const int32_t* __restrict__ p_comp, const uint8_t* __restrict__ c_type,
                           const double* __restrict__ W, const double* __restrict__ cmean,
                           const double* __restrict__ Rp, const float* __restrict__ yhat, float* __restrict__ r,
                           double* __restrict__ acc) {
  double s = 0.0, cnt = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float d = 0.0f;
    const int c = p_comp[p];
    if (c_type[c] == PR_TYPE_SCC && cmean[c] > 0.0) {
      const float y = logf((float)fmax((Rp[p] - W[p]) / cmean[c], 1e-6));
      d = yhat[p] - y;
      s += (double)d * d;
      cnt += 1.0;
    }
    r[p] = d;
  }
  s = group_sum<32>(s);
  cnt = group_sum<32>(cnt);
  if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
    atomicAdd(&acc[0], s);
    atomicAdd(&acc[1], cnt);
  }
}

// dy = 2 r / N
__global__ void mp_scale_k(int32_t n, float* __restrict__ r, const double* __restrict__ acc) {
  const float f = acc[1] > 0.0 ? (float)(2.0 / acc[1]) : 0.0f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    r[p] *= f;
}

// Layer 2 backward, warp per row: dz2 = dy v (g > 0); the direct part
// A2^T dz2 goes to dH1 of the row, the aggregated part B2^T dz2 / d_i to
// dH1 of each internal in-neighbour.
constexpr size_t kMpB2Smem = (size_t)(2 * kMpH * kMpH + kMpH + (kBlock / 32) * kMpH) * sizeof(float);

__global__ void __launch_bounds__(kBlock) mp_b2_k(MpLayout L, const float* __restrict__ dy,
                                                  const float* __restrict__ G, const uint16_t* __restrict__ w16,
                                                  float* __restrict__ dZ2, float* __restrict__ dH1, Ctl* ctl) {
  extern __shared__ float sm[];
  float* A2 = sm;               // [o][k]
  float* B2 = sm + kMpH * kMpH;  // [o][k]
  float* v = B2 + kMpH * kMpH;
  float* stage = v + kMpH;
  for (int t = threadIdx.x; t < kMpH * kMpH; t += blockDim.x) {
    A2[t] = bf2f(w16[kMpA2 + t]);
    B2[t] = bf2f(w16[kMpB2 + t]);
  }
  for (int t = threadIdx.x; t < kMpH; t += blockDim.x) v[t] = bf2f(w16[kMpv + t]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* dz = stage + wib * kMpH;
  const int rows = L.r1 - L.r0;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < rows; i += nw) {
    const int p = L.r0 + (int)i;
    const float d = dy[i];
    const float2 g = *reinterpret_cast<const float2*>(G + (size_t)i * kMpH + 2 * lane);
    const float2 z = make_float2(g.x > 0.0f ? d * v[2 * lane] : 0.0f, g.y > 0.0f ? d * v[2 * lane + 1] : 0.0f);
    *reinterpret_cast<float2*>(dZ2 + (size_t)i * kMpH + 2 * lane) = z;
    if (d == 0.0f || !mp_is_scc(L.p_comp, L.c_type, p)) continue;  // warp-uniform
    dz[2 * lane] = z.x;
    dz[2 * lane + 1] = z.y;
    __syncwarp();
    float h0 = 0.0f, h1 = 0.0f, m0 = 0.0f, m1 = 0.0f;
#pragma unroll 8
    for (int o = 0; o < kMpH; o++) {
      const float zo = dz[o];
      const float2 a = *reinterpret_cast<const float2*>(A2 + o * kMpH + 2 * lane);
      const float2 b = *reinterpret_cast<const float2*>(B2 + o * kMpH + 2 * lane);
      h0 += a.x * zo;
      h1 += a.y * zo;
      m0 += b.x * zo;
      m1 += b.y * zo;
    }
    __syncwarp();
    atomicAdd(&dH1[(size_t)i * kMpH + 2 * lane], h0);
    atomicAdd(&dH1[(size_t)i * kMpH + 2 * lane + 1], h1);
    const int e0 = L.int_ptr[p], e1 = L.int_ptr[p + 1];
    const float inv = e1 > e0 ? 1.0f / (float)(e1 - e0) : 0.0f;
    for (int e = e0; e < e1; e++) {
      const int j = mp_row(L, L.int_idx[e], ctl);
      if (j < 0) continue;
      atomicAdd(&dH1[(size_t)j * kMpH + 2 * lane], m0 * inv);
      atomicAdd(&dH1[(size_t)j * kMpH + 2 * lane + 1], m1 * inv);
    }
  }
}

__global__ void mp_relu_back_k(int64_t count, const float* __restrict__ H1, float* __restrict__ dH1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    if (!(H1[t] > 0.0f)) dH1[t] = 0.0f;
}

// G[o][k] += sum_i D[i][o] X[i][k] and gb[o] += sum_i D[i][o] (gb may be
// null); D is [N][64], X is [N][K] with K in {1, 8, 64}.  Each block keeps
// its outputs in registers over a strided set of 32-row tiles and adds them
// to G once.
constexpr int kMpTile = 32;
__global__ void __launch_bounds__(kBlock) mp_outer_k(int32_t N, const float* __restrict__ D,
                                                     const float* __restrict__ X, int K, float* __restrict__ Gw,
                                                     float* __restrict__ gb) {
  __shared__ float sd[kMpTile * kMpH];
  __shared__ float sx[kMpTile * kMpH];
  const int nout = kMpH * K;
  constexpr int kMaxPer = kMpH * kMpH / kBlock;  // 16
  float acc[kMaxPer];
  float bacc = 0.0f;
#pragma unroll
  for (int j = 0; j < kMaxPer; j++) acc[j] = 0.0f;
  for (int64_t t0 = (int64_t)blockIdx.x * kMpTile; t0 < N; t0 += (int64_t)gridDim.x * kMpTile) {
    const int nr = (int)min((int64_t)kMpTile, N - t0);
    __syncthreads();
    for (int t = threadIdx.x; t < kMpTile * kMpH; t += blockDim.x) {
      const int r = t / kMpH;
      sd[t] = r < nr ? D[(t0 + r) * kMpH + (t % kMpH)] : 0.0f;
    }
    for (int t = threadIdx.x; t < kMpTile * K; t += blockDim.x) {
      const int r = t / K;
      sx[t] = r < nr ? X[(t0 + r) * K + (t % K)] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kMaxPer; j++) {
      const int idx = threadIdx.x + j * kBlock;
      if (idx < nout) {
        const int o = idx / K, k = idx % K;
        float a = 0.0f;
        for (int r = 0; r < kMpTile; r++) a += sd[r * kMpH + o] * sx[r * K + k];
        acc[j] += a;
      }
    }
    if (gb && threadIdx.x < kMpH)
      for (int r = 0; r < kMpTile; r++) bacc += sd[r * kMpH + threadIdx.x];
  }
#pragma unroll
  for (int j = 0; j < kMaxPer; j++) {
    const int idx = threadIdx.x + j * kBlock;
    if (idx < nout) atomicAdd(&Gw[idx], acc[j]);
  }
  if (gb && threadIdx.x < kMpH) atomicAdd(&gb[threadIdx.x], bacc);
}

__global__ void mp_sum_k(int32_t N, const float* __restrict__ x, float* __restrict__ out) {
  float s = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i];
  s = group_sumf<32>(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Adam (bias-corrected), then the bf16 copy; the gradient is cleared
__global__ void mp_adam_k(int count, float* __restrict__ w, float* __restrict__ g, float* __restrict__ m1,
                          float* __restrict__ m2, uint16_t* __restrict__ w16, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    w16[i] = f2bf(w[i]);
    g[i] = 0.0f;
  }
}

__global__ void mp_unperm_k(int32_t n, const int32_t* __restrict__ perm, const float* __restrict__ yp,
                            float* __restrict__ y) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    y[perm[p]] = yp[p];
}

static unsigned mp_grid(int64_t items, int per_block) {
  int64_t g = (items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

static bool g_mp_attr = false;
pr_status mpnn_prepare() {
  if (g_mp_attr) return PR_OK;
  PRGB_CUDA(cudaFuncSetAttribute(mp_l2_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMpL2Smem));
  PRGB_CUDA(cudaFuncSetAttribute(mp_b2_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMpB2Smem));
  g_mp_attr = true;
  return PR_OK;
}

pr_status mpnn_guess(const pr_mpnn_s* M, const pr_partition_s* P, float* yhat, const MpnnInfer& buf, Ctl* ctl,
                     cudaStream_t s) {
  const int32_t n = P->g.n;
  if (n == 0) return PR_OK;
  PRGB_TRY(mpnn_prepare());
  const MpLayout L = mp_layout(P, 0, n);
  const unsigned gn = mp_grid(n, kBlock), gw = mp_grid(n, kBlock / 32);
  PRGB_CUDA(cudaMemsetAsync(buf.dout, 0, (size_t)n * 4, s));
  mp_dout_k<<<gw, kBlock, 0, s>>>(L, buf.dout, ctl);
  PRGB_LAUNCH();
  mp_feat_k<<<gn, kBlock, 0, s>>>(L, buf.dout, buf.X);
  PRGB_LAUNCH();
  mp_l1_k<<<gn, kBlock, 0, s>>>(L, buf.X, M->w16, buf.H1, nullptr, ctl);
  PRGB_LAUNCH();
  mp_l2_k<<<gw, kBlock, kMpL2Smem, s>>>(L, buf.H1, M->w16, yhat, nullptr, nullptr, ctl);
  PRGB_LAUNCH();
  return PR_OK;
}

// R0 = W + exp(clamp(yhat)) mean_C(W) over the rows of SCC c, a CTA per
// component (fixed-order block sum); components above kMpMeanMax vertices
// get R0 = W (the cold start: the guess is not worth a grid-wide sum)
constexpr int kMpMeanMax = 16384;
__global__ void mp_level_r0_k(int32_t c0, const int32_t* __restrict__ c_off, const uint8_t* __restrict__ c_type,
                              const double* __restrict__ W, const float* __restrict__ yhat,
                              double* __restrict__ R0) {
  __shared__ double red[kBlock / 32];
  const int c = c0 + (int)blockIdx.x;
  if (c_type[c] != PR_TYPE_SCC) return;  // block-uniform
  const int o0 = c_off[c], o1 = c_off[c + 1], sz = o1 - o0;
  if (sz > kMpMeanMax) {
    for (int p = o0 + threadIdx.x; p < o1; p += blockDim.x) R0[p] = W[p];
    return;
  }
  double s = 0.0;
  for (int p = o0 + threadIdx.x; p < o1; p += blockDim.x) s += W[p];
  s = group_sum<32>(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  s = group_sum<32>((threadIdx.x & 31) < kBlock / 32 ? red[threadIdx.x & 31] : 0.0);
  const double mean = s / (double)sz;
  for (int p = o0 + threadIdx.x; p < o1; p += blockDim.x)
    R0[p] = W[p] + exp((double)fminf(fmaxf(yhat[p], kMpYMin), kMpYMax)) * mean;
}

pr_status mpnn_level_r0(const pr_partition_s* P, int32_t c0, int32_t c1, const double* W, const float* yhat,
                        double* R0, cudaStream_t s, int64_t* nl) {
  if (c1 <= c0) return PR_OK;
  mp_level_r0_k<<<(unsigned)(c1 - c0), kBlock, 0, s>>>(c0, P->c_off, P->c_type, W, yhat, R0);
  PRGB_LAUNCH();
  ++*nl;
  return PR_OK;
}

// Forward (and with `grad`, backward) over every position of a solved
// partition: yhat by position, the loss, and the gradient added to M->grad.
static pr_status mp_pass(pr_mpnn_s* M, const pr_partition_s* P, double c, const double* u, const double* R,
                         bool grad, float* yhat_pos, double* loss, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  const int32_t n = P->g.n;
  PRGB_TRY(mpnn_prepare());
  double *Rp, *W, *acc, *cmean;
  float *X, *H1, *G, *M1 = nullptr, *M2 = nullptr, *yh, *dy;
  int32_t* dout;
  PRGB_TRY(tmp.alloc(&Rp, n));
  PRGB_TRY(tmp.alloc(&W, n));
  PRGB_TRY(tmp.alloc(&cmean, (size_t)P->n_comp + 1));
  PRGB_TRY(tmp.alloc(&dout, (size_t)n + 1));
  PRGB_TRY(tmp.alloc(&acc, 2));
  PRGB_TRY(tmp.alloc(&X, (size_t)n * kMpF0));
  PRGB_TRY(tmp.alloc(&H1, (size_t)n * kMpH));
  PRGB_TRY(tmp.alloc(&G, (size_t)n * kMpH));
  PRGB_TRY(tmp.alloc(&yh, n));
  PRGB_TRY(tmp.alloc(&dy, n));
  if (grad) {
    PRGB_TRY(tmp.alloc(&M1, (size_t)n * kMpF0));
    PRGB_TRY(tmp.alloc(&M2, (size_t)n * kMpH));
  }
  PRGB_CUDA(cudaMemsetAsync(acc, 0, 16, s));
  const MpLayout L = mp_layout(P, 0, n);
  const unsigned gn = mp_grid(n, kBlock), gw = mp_grid(n, kBlock / 32);
  mp_rpos_k<<<gn, kBlock, 0, s>>>(n, P->perm, R, Rp);
  PRGB_LAUNCH();
  mp_w_k<<<gn, kBlock, 0, s>>>(n, P->perm, u, Rp, P->ext_ptr, P->ext_idx, P->p_inv, c, W);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaMemsetAsync(cmean, 0, ((size_t)P->n_comp + 1) * 8, s));
  mp_cmean_k<<<mp_grid(P->n_comp, kBlock / 32), kBlock, 0, s>>>(P->n_comp, P->c_off, P->c_type, W, cmean);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaMemsetAsync(dout, 0, ((size_t)n + 1) * 4, s));
  mp_dout_k<<<gw, kBlock, 0, s>>>(L, dout, ctl);
  PRGB_LAUNCH();
  mp_feat_k<<<gn, kBlock, 0, s>>>(L, dout, X);
  PRGB_LAUNCH();
  mp_l1_k<<<gn, kBlock, 0, s>>>(L, X, M->w16, H1, M1, ctl);
  PRGB_LAUNCH();
  mp_l2_k<<<gw, kBlock, kMpL2Smem, s>>>(L, H1, M->w16, yh, G, M2, ctl);
  PRGB_LAUNCH();
  mp_resid_k<<<gn, kBlock, 0, s>>>(n, P->p_comp, P->c_type, W, cmean, Rp, yh, dy, acc);
  PRGB_LAUNCH();
  if (yhat_pos) PRGB_CUDA(cudaMemcpyAsync(yhat_pos, yh, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  if (grad) {
    float *dZ2, *dH1;
    PRGB_TRY(tmp.alloc(&dZ2, (size_t)n * kMpH));
    PRGB_TRY(tmp.alloc(&dH1, (size_t)n * kMpH));
    PRGB_CUDA(cudaMemsetAsync(dH1, 0, (size_t)n * kMpH * 4, s));
    mp_scale_k<<<gn, kBlock, 0, s>>>(n, dy, acc);
    PRGB_LAUNCH();
    mp_b2_k<<<gw, kBlock, kMpB2Smem, s>>>(L, dy, G, M->w16, dZ2, dH1, ctl);
    PRGB_LAUNCH();
    mp_relu_back_k<<<mp_grid((int64_t)n * kMpH, kBlock), kBlock, 0, s>>>((int64_t)n * kMpH, H1, dH1);
    PRGB_LAUNCH();
    const unsigned go = mp_grid(n, kMpTile);
    float* g = M->grad;
    mp_outer_k<<<go, kBlock, 0, s>>>(n, dZ2, H1, kMpH, g + kMpA2, g + kMpb2);
    PRGB_LAUNCH();
    mp_outer_k<<<go, kBlock, 0, s>>>(n, dZ2, M2, kMpH, g + kMpB2, nullptr);
    PRGB_LAUNCH();
    mp_outer_k<<<go, kBlock, 0, s>>>(n, G, dy, 1, g + kMpv, nullptr);
    PRGB_LAUNCH();
    mp_sum_k<<<gn, kBlock, 0, s>>>(n, dy, g + kMpb3);
    PRGB_LAUNCH();
    mp_outer_k<<<go, kBlock, 0, s>>>(n, dH1, X, kMpF0, g + kMpA1, g + kMpb1);
    PRGB_LAUNCH();
    mp_outer_k<<<go, kBlock, 0, s>>>(n, dH1, M1, kMpF0, g + kMpB1, nullptr);
    PRGB_LAUNCH();
  }
  double h[2] = {0.0, 0.0};
  PRGB_CUDA(cudaMemcpyAsync(h, acc, 16, cudaMemcpyDeviceToHost, s));
  int err = 0;
  PRGB_CUDA(cudaMemcpyAsync(&err, &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (err) return (pr_status)err;
  if (loss) *loss = h[1] > 0.0 ? h[0] / h[1] : 0.0;
  return PR_OK;
}

// splitmix64 (Steele, Lea and Flood, 2014): the seeded initial weights
static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace prgb

using namespace prgb;

extern "C" {

int64_t pr_mpnn_param_count(void) { return kMpParams; }

static pr_status pr_mpnn_create_body(uint64_t seed, void* stream, pr_mpnn** out) {
  if (!out) return PR_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  pr_mpnn_s* M = new (std::nothrow) pr_mpnn_s;
  if (!M) return PR_ENOMEM;
  M->stream = s;
  static std::atomic<uint64_t> next_uid{1};
  M->uid = next_uid.fetch_add(1, std::memory_order_relaxed);
  M->keep = new (std::nothrow) Arena(s);
  if (!M->keep) {
    delete M;
    return PR_ENOMEM;
  }
  pr_status st = PR_OK;
  if (st == PR_OK) st = M->keep->alloc(&M->master, kMpParams);
  if (st == PR_OK) st = M->keep->alloc(&M->m1, kMpParams);
  if (st == PR_OK) st = M->keep->alloc(&M->m2, kMpParams);
  if (st == PR_OK) st = M->keep->alloc(&M->grad, kMpParams);
  if (st == PR_OK) st = M->keep->alloc(&M->w16, kMpParams);
  if (st == PR_OK) {
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, b3 = 1
    std::vector<float> h(kMpParams, 0.0f);
    uint64_t x = seed;
    auto fill = [&](int off, int outs, int fan_in) {
      const float a = 1.0f / sqrtf((float)fan_in);
      for (int t = 0; t < outs * fan_in; t++) {
        const double r = (double)(splitmix64(&x) >> 11) * (1.0 / 9007199254740992.0);
        h[off + t] = (float)((2.0 * r - 1.0) * a);
      }
    };
    fill(kMpA1, kMpH, kMpF0);
    fill(kMpB1, kMpH, kMpF0);
    fill(kMpA2, kMpH, kMpH);
    fill(kMpB2, kMpH, kMpH);
    fill(kMpv, 1, kMpH);
    h[kMpb3] = 1.0f;
    if (cudaMemcpyAsync(M->master, h.data(), kMpParams * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(M->m1, 0, kMpParams * 4, s) != cudaSuccess ||
        cudaMemsetAsync(M->m2, 0, kMpParams * 4, s) != cudaSuccess ||
        cudaMemsetAsync(M->grad, 0, kMpParams * 4, s) != cudaSuccess)
      st = PR_ECUDA;
    if (st == PR_OK) {
      mp_to_bf16_k<<<mp_grid(kMpParams, kBlock), kBlock, 0, s>>>(kMpParams, M->master, M->w16);
      count_launch();
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = PR_ECUDA;
    }
  }
  if (st != PR_OK) {
    delete M->keep;
    delete M;
    return st;
  }
  *out = M;
  return PR_OK;
}

pr_status pr_mpnn_create(uint64_t seed, void* stream, pr_mpnn** out) {
  return prgb::note_status(pr_mpnn_create_body(seed, stream, out));
}

void pr_mpnn_destroy(pr_mpnn* M) {
  if (!M) return;
  delete M->keep;
  delete M;
}

static pr_status pr_mpnn_get_params_body(const pr_mpnn* M, float* host, int64_t count) {
  if (!M || !host || count != kMpParams) return PR_EINVAL;
  PRGB_CUDA(cudaMemcpyAsync(host, M->master, kMpParams * 4, cudaMemcpyDeviceToHost, M->stream));
  PRGB_CUDA(cudaStreamSynchronize(M->stream));
  return PR_OK;
}

pr_status pr_mpnn_get_params(const pr_mpnn* M, float* host, int64_t count) {
  return prgb::note_status(pr_mpnn_get_params_body(M, host, count));
}

static pr_status pr_mpnn_set_params_body(pr_mpnn* M, const float* host, int64_t count) {
  if (!M || !host || count != kMpParams) return PR_EINVAL;
  cudaStream_t s = M->stream;
  PRGB_CUDA(cudaMemcpyAsync(M->master, host, kMpParams * 4, cudaMemcpyHostToDevice, s));
  PRGB_CUDA(cudaMemsetAsync(M->m1, 0, kMpParams * 4, s));
  PRGB_CUDA(cudaMemsetAsync(M->m2, 0, kMpParams * 4, s));
  PRGB_CUDA(cudaMemsetAsync(M->grad, 0, kMpParams * 4, s));
  M->step = 0;
  M->version++;
  mp_to_bf16_k<<<mp_grid(kMpParams, kBlock), kBlock, 0, s>>>(kMpParams, M->master, M->w16);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaStreamSynchronize(s));
  return PR_OK;
}

pr_status pr_mpnn_set_params(pr_mpnn* M, const float* host, int64_t count) {
  return prgb::note_status(pr_mpnn_set_params_body(M, host, count));
}

static pr_status mp_check(const pr_mpnn* M, const pr_partition* part, double c, const double* u, const double* R) {
  if (!M || !part) return PR_EINVAL;
  if (!(c > 0.0 && c < 1.0)) return PR_EINVAL;
  if (part->g.n > 0 && (!u || !R)) return PR_EINVAL;
  return PR_OK;
}

static pr_status pr_mpnn_predict_body(const pr_mpnn* M, const pr_partition* part, double c, const double* u,
                                      const double* R, float* yhat, double* loss, void* stream) {
  PRGB_TRY(mp_check(M, part, c, u, R));
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = part->g.n;
  Arena tmp(s);
  Ctl* ctl = nullptr;
  float* yp = nullptr;
  PRGB_TRY(tmp.alloc(&ctl, 1));
  PRGB_TRY(tmp.alloc(&yp, (size_t)n + 1));
  PRGB_TRY(init_ctl(ctl, s));
  PRGB_TRY(mp_pass(const_cast<pr_mpnn*>(M), part, c, u, R, false, yp, loss, tmp, ctl));
  if (yhat && n > 0) {
    mp_unperm_k<<<mp_grid(n, kBlock), kBlock, 0, s>>>(n, part->perm, yp, yhat);
    PRGB_LAUNCH();
    PRGB_CUDA(cudaStreamSynchronize(s));
  }
  return PR_OK;
}

pr_status pr_mpnn_predict(const pr_mpnn* M, const pr_partition* part, double c, const double* u, const double* R,
                          float* yhat, double* loss, void* stream) {
  return prgb::note_status(pr_mpnn_predict_body(M, part, c, u, R, yhat, loss, stream));
}

static pr_status pr_mpnn_loss_grad_body(pr_mpnn* M, const pr_partition* part, double c, const double* u,
                                        const double* R, float* grad_host, double* loss, void* stream) {
  PRGB_TRY(mp_check(M, part, c, u, R));
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp(s);
  Ctl* ctl = nullptr;
  PRGB_TRY(tmp.alloc(&ctl, 1));
  PRGB_TRY(init_ctl(ctl, s));
  PRGB_CUDA(cudaMemsetAsync(M->grad, 0, kMpParams * 4, s));
  PRGB_TRY(mp_pass(M, part, c, u, R, true, nullptr, loss, tmp, ctl));
  if (grad_host) {
    PRGB_CUDA(cudaMemcpyAsync(grad_host, M->grad, kMpParams * 4, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
  }
  PRGB_CUDA(cudaMemsetAsync(M->grad, 0, kMpParams * 4, s));
  return PR_OK;
}

pr_status pr_mpnn_loss_grad(pr_mpnn* M, const pr_partition* part, double c, const double* u, const double* R,
                            float* grad_host, double* loss, void* stream) {
  return prgb::note_status(pr_mpnn_loss_grad_body(M, part, c, u, R, grad_host, loss, stream));
}

static pr_status pr_mpnn_train_step_body(pr_mpnn* M, const pr_partition* part, double c, const double* u,
                                         const double* R, float lr, double* loss, void* stream) {
  PRGB_TRY(mp_check(M, part, c, u, R));
  if (!(lr > 0.0f)) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp(s);
  Ctl* ctl = nullptr;
  PRGB_TRY(tmp.alloc(&ctl, 1));
  PRGB_TRY(init_ctl(ctl, s));
  PRGB_CUDA(cudaMemsetAsync(M->grad, 0, kMpParams * 4, s));
  PRGB_TRY(mp_pass(M, part, c, u, R, true, nullptr, loss, tmp, ctl));
  M->step++;
  M->version++;
  const float c1 = 1.0f - powf(0.9f, (float)M->step), c2 = 1.0f - powf(0.999f, (float)M->step);
  mp_adam_k<<<mp_grid(kMpParams, kBlock), kBlock, 0, s>>>(kMpParams, M->master, M->grad, M->m1, M->m2, M->w16, lr,
                                                          c1, c2);
  PRGB_LAUNCH();
  // later solves on other streams see the new weights
  PRGB_CUDA(cudaStreamSynchronize(s));
  return PR_OK;
}

pr_status pr_mpnn_train_step(pr_mpnn* M, const pr_partition* part, double c, const double* u, const double* R,
                             float lr, double* loss, void* stream) {
  return prgb::note_status(pr_mpnn_train_step_body(M, part, c, u, R, lr, loss, stream));
}

}  // extern "C"
