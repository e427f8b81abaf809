// mpnn.cuh -- the learned warm start of the SCC power series: a two-layer
// message-passing network over each SCC's internal in-edges that guesses
// each row's amplification (R_i - W_i) / mean_C(W) (mpnn.cu).
#pragma once

#include "common.cuh"

namespace prgb {

constexpr int kMpF0 = 8;  // input features per vertex
constexpr int kMpH = 64;  // hidden width
// parameter vector (float32 masters, bf16 copies for the forward pass):
// A1[64][8], B1[64][8], b1[64], A2[64][64], B2[64][64], b2[64], v[64], b3
constexpr int kMpA1 = 0;
constexpr int kMpB1 = kMpA1 + kMpH * kMpF0;
constexpr int kMpb1 = kMpB1 + kMpH * kMpF0;
constexpr int kMpA2 = kMpb1 + kMpH;
constexpr int kMpB2 = kMpA2 + kMpH * kMpH;
constexpr int kMpb2 = kMpB2 + kMpH * kMpH;
constexpr int kMpv = kMpb2 + kMpH;
constexpr int kMpb3 = kMpv + kMpH;
constexpr int kMpParams = kMpb3 + 1;

// the guess's clamp: R0 = W + exp(clamp(yhat, kMpYMin, kMpYMax)) mean_C(W)
constexpr float kMpYMin = -14.0f;
constexpr float kMpYMax = 9.0f;

// scratch of one inference pass over every row of the permuted layout
struct MpnnInfer {
  float* X = nullptr;      // [n][8]
  float* H1 = nullptr;     // [n][64]
  int32_t* dout = nullptr; // [n] internal out-degree
};

// one-time kernel attributes of the network's kernels (call before any
// stream capture that launches them)
pr_status mpnn_prepare();

// yhat by position for every SCC row (0 elsewhere): the network's guess of
// log of the row's amplification, from the structure only.  Launches only.
pr_status mpnn_guess(const pr_mpnn_s* M, const pr_partition_s* P, float* yhat, const MpnnInfer& buf, Ctl* ctl,
                     cudaStream_t s);

// R0 of the SCC rows of components [c0, c1) from the level's W and yhat
// (a CTA per component; R0 = W above 16,384 vertices).  One launch
// (capturable).
pr_status mpnn_level_r0(const pr_partition_s* P, int32_t c0, int32_t c1, const double* W, const float* yhat,
                        double* R0, cudaStream_t s, int64_t* nl);

}  // namespace prgb

// the opaque model of the C ABI
struct pr_mpnn_s {
  cudaStream_t stream = nullptr;
  prgb::Arena* keep = nullptr;
  float* master = nullptr;  // [kMpParams] float32 weights
  float* m1 = nullptr;      // Adam moments
  float* m2 = nullptr;
  float* grad = nullptr;    // [kMpParams] accumulated gradient
  uint16_t* w16 = nullptr;  // [kMpParams] bf16 copy used by the forward pass
  int64_t step = 0;
  // process-unique id (never reused): a captured solve that runs this
  // network is matched by it, not by the handle's address, which a later
  // model may receive once this one is destroyed
  uint64_t uid = 0;
  uint64_t version = 0;  // bumped by every change of the weights
};
