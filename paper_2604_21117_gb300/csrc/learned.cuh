// Learned leaf predictor: device-side model evaluation shared by the fitting,
// training, error-bound and search kernels.
//
// The paper has no learned component.  A small fp32 model predicts the leaf
// of a key directly, so the search can skip the inner levels; the model's
// maximum error over the stored keys (computed by the same device code)
// bounds a window of leaves, whose boundaries are checked with exact integer
// compares against the leaves' largest keys; a query whose leaf is not
// proven to lie in the window takes the plain level-wise descent, so results
// are always those of the plain tree.
//
// Models (all arithmetic in fp32 unless stated; the fp32 steps below are the
// exact operations the CPU oracle reproduces):
//   PL  (piecewise linear, S segments): b_s = key of rank floor(s*n/S);
//       segment of q = largest s with b_s <= q (0 below b_0);
//       x = fp32(fp64(q - b_s)) * inv_w_s,  inv_w_s = fp32(1 / fp64(b_{s+1} - b_s));
//       pred = fp32(fp32(slope_s * x) + icpt_s), separately rounded.
//   MLP (1 -> 32 -> 32 -> 1, ReLU) on a rank coordinate (a two-stage model):
//       the first stage is kMlpStage1 breakpoints b_s at key quantiles, as the
//       PL model's; x = fp32(fp32(s) + min(fp32(fp64(q - b_s)) * inv_w_s, 1))
//       * (1 / kMlpStage1), so that x follows the key's rank whatever the key
//       distribution; pred = (w3 . relu(W2 relu(W1 x + b1) + b2) + b3) * (L - 1).
//   leaf_hat = rint(clamp(pred, 0, L - 1)).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace btgb {

constexpr int kMlpH = 32;
constexpr uint32_t kMlpStage1 = 64;  // breakpoints of the MLP's first stage
constexpr int kMlpParams = kMlpH + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 1153
// parameter offsets: W1[32], b1[32], W2[32][32] (row = output unit), b2[32], w3[32], b3
constexpr int kOffW1 = 0, kOffB1 = 32, kOffW2 = 64, kOffB2 = 64 + 1024, kOffW3 = 64 + 1024 + 32,
              kOffB3 = 64 + 1024 + 64;

enum ModelKind : int { kModelNone = 0, kModelPL = 1, kModelMLP = 2 };

// The error bound is kept per range of predicted leaf: range r covers
// leaf_hat in [r*L/kErrRanges, (r+1)*L/kErrRanges).  A stored key with
// prediction leaf_hat lies within errs[range(leaf_hat)] leaves of it.
constexpr uint32_t kErrRanges = 256;

__host__ __device__ __forceinline__ uint32_t err_range(uint32_t hat, uint32_t L)
{
    return static_cast<uint32_t>((static_cast<uint64_t>(hat) * kErrRanges) / L);
}

// Everything the search kernel needs to use a model, passed by value.
struct ModelDev {
    int kind;
    uint32_t segments;      // PL
    uint32_t err;           // max |leaf_hat - leaf| over the stored keys
    const uint32_t *errs;   // the same maximum per range of leaf_hat (kErrRanges ranges)
    uint32_t leaves;        // L
    const uint64_t *b;      // PL breakpoints (as uint64 whatever the key width)
    const float *inv_w;     // PL
    const float *slope;     // PL
    const float *icpt;      // PL
    const float *mlp;       // MLP parameters
    const void *leaf_max;   // largest key of every leaf (key width)
    uint64_t kmin, kmax;
    float inv_range;        // MLP
};

__device__ __forceinline__ int pl_segment(const uint64_t *b, uint32_t S, uint64_t q)
{
    // largest s with b[s] <= q, 0 if q < b[0]
    int lo = 0, hi = static_cast<int>(S) - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float pl_predict(const uint64_t *b, const float *inv_w, const float *slope,
                                            const float *icpt, uint32_t S, uint64_t q)
{
    const int s = pl_segment(b, S, q);
    const uint64_t diff = q >= b[s] ? q - b[s] : 0ull;
    const float x = __fmul_rn(__double2float_rn(__ull2double_rn(diff)), inv_w[s]);
    return __fadd_rn(__fmul_rn(slope[s], x), icpt[s]);
}

// The MLP's input: the rank coordinate of q from the first stage's
// breakpoints (b, inv_w: kMlpStage1 entries, any address space).
__device__ __forceinline__ float mlp_x_rank(const uint64_t *b, const float *inv_w, uint64_t q)
{
    const int s = pl_segment(b, kMlpStage1, q);
    const uint64_t diff = q >= b[s] ? q - b[s] : 0ull;
    const float u = fminf(__fmul_rn(__double2float_rn(__ull2double_rn(diff)), inv_w[s]), 1.0f);
    return __fmul_rn(__fadd_rn(static_cast<float>(s), u), 1.0f / static_cast<float>(kMlpStage1));
}

__device__ __forceinline__ float mlp_x(uint64_t q, uint64_t kmin, uint64_t kmax, float inv_range)
{
    const uint64_t c = q < kmin ? kmin : (q > kmax ? kmax : q);
    return __fmul_rn(__double2float_rn(__ull2double_rn(c - kmin)), inv_range);
}

// Network output for input x (parameters p, any address space).
__device__ __forceinline__ float mlp_forward(const float *p, float x)
{
    float h1[kMlpH];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) h1[j] = fmaxf(fmaf(p[kOffW1 + j], x, p[kOffB1 + j]), 0.0f);
    float y = p[kOffB3];
#pragma unroll 4
    for (int j = 0; j < kMlpH; ++j) {
        float z = p[kOffB2 + j];
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) z = fmaf(p[kOffW2 + j * kMlpH + k], h1[k], z);
        y = fmaf(p[kOffW3 + j], fmaxf(z, 0.0f), y);
    }
    return y;
}

__device__ __forceinline__ uint32_t leaf_from_pred(float pred, uint32_t L)
{
    const float hiv = static_cast<float>(L - 1);
    pred = fminf(fmaxf(pred, 0.0f), hiv);
    return static_cast<uint32_t>(__float2int_rn(pred));
}

// Predicted leaf of q; PL parameters may live in shared memory (pointers given).
__device__ __forceinline__ uint32_t model_leaf(const ModelDev &m, const uint64_t *b, const float *inv_w,
                                               const float *slope, const float *icpt, const float *mlp,
                                               uint64_t q)
{
    if (m.kind == kModelPL) return leaf_from_pred(pl_predict(b, inv_w, slope, icpt, m.segments, q), m.leaves);
    const float y = mlp_forward(mlp, mlp_x_rank(b, inv_w, q));
    return leaf_from_pred(__fmul_rn(y, static_cast<float>(m.leaves - 1)), m.leaves);
}

// Leaf holding the stored key of rank i under the even bulk load: leaf j
// holds base + (j < rem) keys, the larger leaves first.
__device__ __forceinline__ void rank_to_leaf(uint64_t i, uint64_t base, uint64_t rem, uint64_t &leaf,
                                             uint64_t &slot)
{
    const uint64_t big = rem * (base + 1);
    if (i < big) {
        leaf = i / (base + 1);
        slot = i - leaf * (base + 1);
    } else {
        leaf = rem + (i - big) / base;
        slot = i - big - (leaf - rem) * base;
    }
}

// splitmix64 (Steele, Lea & Flood, "Fast Splittable Pseudorandom Number
// Generators", OOPSLA 2014): the output function applied to a counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace btgb
