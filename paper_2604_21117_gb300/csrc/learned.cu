// Learned leaf predictor: fitting (PL), training (MLP), error bound, API.
//
// Everything here runs on the GPU: the training pairs are the stored keys
// with the index of the leaf that holds them, read straight from the built
// tree's leaf blocks; the PL model is a per-segment least-squares fit
// (fp64 sums, fp32 parameters); the MLP is trained by this file's own
// forward/backward kernel and an Adam step kernel; the maximum error over
// all stored keys is computed by the same device prediction code that the
// search uses.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "bt_internal.h"

namespace btgb {

static inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

template <typename K>
__device__ __forceinline__ uint64_t key_of_rank(const DevTree &t, uint64_t i, uint64_t &leaf)
{
    const int lv = t.height - 1;
    uint64_t slot;
    rank_to_leaf(i, t.cbase[lv], t.crem[lv], leaf, slot);
    return static_cast<uint64_t>(static_cast<const K *>(t.keys[lv])[leaf * t.m + slot]);
}

template <typename K>
__global__ void k_leaf_max(const DevTree t, K *__restrict__ leaf_max)
{
    const int lv = t.height - 1;
    const uint64_t L = t.nodes[lv];
    const K *keys = static_cast<const K *>(t.keys[lv]);
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < L;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t cnt = t.cbase[lv] + (j < t.crem[lv] ? 1u : 0u);
        leaf_max[j] = keys[j * t.m + cnt - 1];
    }
}

// ------------------------------------------------------------- PL fit

template <typename K>
__global__ void k_pl_breaks(const DevTree t, uint32_t S, uint64_t *__restrict__ b, float *__restrict__ inv_w)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const uint64_t n = t.cbase[t.height - 1] * t.nodes[t.height - 1] + t.crem[t.height - 1];
    uint64_t leaf;
    const uint64_t bs = key_of_rank<K>(t, static_cast<uint64_t>(s) * n / S, leaf);
    uint64_t next;
    if (s + 1 < S)
        next = key_of_rank<K>(t, static_cast<uint64_t>(s + 1) * n / S, leaf);
    else
        next = (t.kmax == ~0ull) ? t.kmax : t.kmax + 1;
    uint64_t width = next > bs ? next - bs : 1ull;
    b[s] = bs;
    inv_w[s] = __double2float_rn(1.0 / __ull2double_rn(width));
}

// Per-segment sums (count, x, y, xx, xy) in fp64 over every stored key.
template <typename K>
__global__ void k_pl_sums(const DevTree t, uint32_t S, const uint64_t *__restrict__ b,
                          const float *__restrict__ inv_w, double *__restrict__ sums)
{
    const uint64_t n = t.cbase[t.height - 1] * t.nodes[t.height - 1] + t.crem[t.height - 1];
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    int cur = -1;
    double c = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        // segment of the key of rank i: largest s with floor(s*n/S) <= i
        const int s = static_cast<int>(((i + 1) * S - 1) / n);
        if (s != cur) {
            if (cur >= 0) {
                double *o = sums + 5 * cur;
                atomicAdd(o + 0, c);
                atomicAdd(o + 1, sx);
                atomicAdd(o + 2, sy);
                atomicAdd(o + 3, sxx);
                atomicAdd(o + 4, sxy);
            }
            cur = s;
            c = sx = sy = sxx = sxy = 0;
        }
        uint64_t leaf;
        const uint64_t key = key_of_rank<K>(t, i, leaf);
        const uint64_t diff = key >= b[s] ? key - b[s] : 0ull;
        const double x = static_cast<double>(__fmul_rn(__double2float_rn(__ull2double_rn(diff)), inv_w[s]));
        const double y = static_cast<double>(leaf);
        c += 1.0;
        sx += x;
        sy += y;
        sxx += x * x;
        sxy += x * y;
    }
    if (cur >= 0) {
        double *o = sums + 5 * cur;
        atomicAdd(o + 0, c);
        atomicAdd(o + 1, sx);
        atomicAdd(o + 2, sy);
        atomicAdd(o + 3, sxx);
        atomicAdd(o + 4, sxy);
    }
}

// Closed-form least squares per segment; a segment whose x values do not
// vary gets a flat line at the mean leaf.
__global__ void k_pl_solve(uint32_t S, const double *__restrict__ sums, float *__restrict__ slope,
                           float *__restrict__ icpt)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double c = sums[5 * s], sx = sums[5 * s + 1], sy = sums[5 * s + 2], sxx = sums[5 * s + 3],
                 sxy = sums[5 * s + 4];
    double a = 0.0, k = (c > 0) ? sy / c : 0.0;
    const double den = c * sxx - sx * sx;
    if (c >= 2.0 && den > 1e-12 * c * sxx) {
        a = (c * sxy - sx * sy) / den;
        k = (sy - a * sx) / c;
    }
    slope[s] = __double2float_rn(a);
    icpt[s] = __double2float_rn(k);
}

// ------------------------------------------------------- MLP training

constexpr int kMlpBlock = 128;
constexpr int kMlpPad = kMlpH + 1;

struct MlpSmem {
    float p[kMlpParams];
    float x[kMlpBlock];
    float dy[kMlpBlock];
    float h1[kMlpBlock][kMlpPad];
    float h2[kMlpBlock][kMlpPad];
    float dz1[kMlpBlock][kMlpPad];
    float dz2[kMlpBlock][kMlpPad];
    float red[kMlpBlock / 32];
};

// Mean-squared-error gradient of the MLP over `count` samples, added into
// grad[] and loss[0].  SAMPLE: the samples are stored keys of ranks drawn by
// splitmix64(seed, step, i) with target leaf / (L - 1); otherwise x[] and
// t[] are given.
template <bool SAMPLE, typename K>
__global__ void __launch_bounds__(kMlpBlock) k_mlp_grad(const float *__restrict__ params,
                                                        const float *__restrict__ xs, const float *__restrict__ ts,
                                                        uint32_t count, const DevTree t, ModelDev md, uint64_t seed,
                                                        uint32_t step, float *__restrict__ grad,
                                                        float *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < kMlpParams; i += blockDim.x) S.p[i] = params[i];
    __syncthreads();
    const uint32_t i = blockIdx.x * kMlpBlock + tid;
    const bool valid = i < count;
    float x = 0.0f, tv = 0.0f;
    if (valid) {
        if (SAMPLE) {
            const int lv = t.height - 1;
            const uint64_t n = t.cbase[lv] * t.nodes[lv] + t.crem[lv];
            const uint64_t r = splitmix64(seed ^ ((static_cast<uint64_t>(step) << 32) | i)) % n;
            uint64_t leaf;
            const uint64_t key = key_of_rank<K>(t, r, leaf);
            x = mlp_x_rank(md.b, md.inv_w, key);
            tv = md.leaves > 1 ? __fdiv_rn(static_cast<float>(leaf), static_cast<float>(md.leaves - 1)) : 0.0f;
        } else {
            x = xs[i];
            tv = ts[i];
        }
    }
    // forward
    float z1[kMlpH], z2[kMlpH];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) z1[j] = fmaf(S.p[kOffW1 + j], x, S.p[kOffB1 + j]);
    float y = S.p[kOffB3];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float z = S.p[kOffB2 + j];
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) z = fmaf(S.p[kOffW2 + j * kMlpH + k], fmaxf(z1[k], 0.0f), z);
        z2[j] = z;
        y = fmaf(S.p[kOffW3 + j], fmaxf(z, 0.0f), y);
    }
    const float inv_n = 1.0f / static_cast<float>(count);
    const float e = valid ? (y - tv) : 0.0f;
    const float dy = 2.0f * e * inv_n;
    // backward
    float dh1[kMlpH];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) dh1[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        const float dz = (z2[j] > 0.0f) ? dy * S.p[kOffW3 + j] : 0.0f;
        S.dz2[tid][j] = dz;
        S.h2[tid][j] = fmaxf(z2[j], 0.0f);
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) dh1[k] = fmaf(S.p[kOffW2 + j * kMlpH + k], dz, dh1[k]);
    }
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        S.h1[tid][k] = fmaxf(z1[k], 0.0f);
        S.dz1[tid][k] = (z1[k] > 0.0f) ? dh1[k] : 0.0f;
    }
    S.x[tid] = x;
    S.dy[tid] = dy;
    // loss (mean squared error), reduced over the block
    float l2 = e * e * inv_n;
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = l2;
    __syncthreads();
    if (tid == 0) {
        float s = 0.0f;
        for (int w = 0; w < kMlpBlock / 32; ++w) s += S.red[w];
        atomicAdd(loss, s);
    }
    // parameter gradients summed over the block's samples
    for (int q = tid; q < kMlpParams; q += blockDim.x) {
        float g = 0.0f;
        if (q < kOffB1) {
            for (int s = 0; s < kMlpBlock; ++s) g = fmaf(S.dz1[s][q], S.x[s], g);
        } else if (q < kOffW2) {
            for (int s = 0; s < kMlpBlock; ++s) g += S.dz1[s][q - kOffB1];
        } else if (q < kOffB2) {
            const int j = (q - kOffW2) / kMlpH, k = (q - kOffW2) % kMlpH;
            for (int s = 0; s < kMlpBlock; ++s) g = fmaf(S.dz2[s][j], S.h1[s][k], g);
        } else if (q < kOffW3) {
            for (int s = 0; s < kMlpBlock; ++s) g += S.dz2[s][q - kOffB2];
        } else if (q < kOffB3) {
            for (int s = 0; s < kMlpBlock; ++s) g = fmaf(S.dy[s], S.h2[s][q - kOffW3], g);
        } else {
            for (int s = 0; s < kMlpBlock; ++s) g += S.dy[s];
        }
        atomicAdd(grad + q, g);
    }
}

// One Adam step (Kingma & Ba 2015) on every parameter; clears the gradient.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m1, float *__restrict__ m2,
                       uint32_t step, float lr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float c1 = 1.0f - powf(b1, static_cast<float>(step + 1));
    const float c2 = 1.0f - powf(b2, static_cast<float>(step + 1));
    p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    g[i] = 0.0f;
}

// ------------------------------------------------------ error bound

// Largest |leaf_hat - leaf| over every stored key, overall (err[0]) and per
// range of leaf_hat (errs[]), by the same prediction code the search uses.
template <typename K>
__global__ void k_model_err(const DevTree t, ModelDev md, uint32_t *__restrict__ err, uint32_t *__restrict__ errs)
{
    __shared__ uint32_t se[kErrRanges];
    for (uint32_t i = threadIdx.x; i < kErrRanges; i += blockDim.x) se[i] = 0;
    __syncthreads();
    const int lv = t.height - 1;
    const uint64_t n = t.cbase[lv] * t.nodes[lv] + t.crem[lv];
    uint32_t e = 0;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t leaf;
        const uint64_t key = key_of_rank<K>(t, i, leaf);
        const uint32_t hat = model_leaf(md, md.b, md.inv_w, md.slope, md.icpt, md.mlp, key);
        const uint32_t d = hat > leaf ? hat - static_cast<uint32_t>(leaf) : static_cast<uint32_t>(leaf) - hat;
        e = d > e ? d : e;
        if (d) atomicMax(&se[err_range(hat, md.leaves)], d);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    if ((threadIdx.x & 31) == 0) atomicMax(err, e);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kErrRanges; i += blockDim.x)
        if (se[i]) atomicMax(errs + i, se[i]);
}

static bt_status cuda_fail(const char *what, cudaError_t e)
{
    set_error_detail(what, e);
    return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
}

template <typename K>
static bt_status train_impl(const bt_tree *tree, const bt_learn_opts *o, cudaStream_t s, bt_model *mdl)
{
    const DevTree &t = tree->dev;
    ModelDev &md = mdl->dev;
    const uint64_t n = tree->info.n;
    const uint64_t L = t.nodes[t.height - 1];
    const uint32_t grid = 1024;
    cudaError_t e;
    k_leaf_max<K><<<grid, 256, 0, s>>>(t, static_cast<K *>(const_cast<void *>(md.leaf_max)));
    if (md.kind == kModelPL) {
        const uint32_t S = md.segments;
        double *sums = reinterpret_cast<double *>(const_cast<float *>(md.icpt) + S);
        sums = reinterpret_cast<double *>(a256(reinterpret_cast<uintptr_t>(sums)));
        e = cudaMemsetAsync(sums, 0, static_cast<size_t>(S) * 5 * sizeof(double), s);
        if (e != cudaSuccess) return cuda_fail("memset of fit sums", e);
        k_pl_breaks<K><<<(S + 255) / 256, 256, 0, s>>>(t, S, const_cast<uint64_t *>(md.b),
                                                      const_cast<float *>(md.inv_w));
        k_pl_sums<K><<<grid, 256, 0, s>>>(t, S, md.b, md.inv_w, sums);
        k_pl_solve<<<(S + 255) / 256, 256, 0, s>>>(S, sums, const_cast<float *>(md.slope),
                                                   const_cast<float *>(md.icpt));
    } else {
        // the first stage: breakpoints at key quantiles, as the PL model's
        k_pl_breaks<K><<<1, 256, 0, s>>>(t, kMlpStage1, const_cast<uint64_t *>(md.b), const_cast<float *>(md.inv_w));
        float *p = const_cast<float *>(md.mlp);
        float *g = p + kMlpParams, *m1 = g + kMlpParams, *m2 = m1 + kMlpParams, *loss = m2 + kMlpParams;
        e = cudaMemcpyAsync(p, o->h_init, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, (3 * kMlpParams + 1) * sizeof(float), s);
        if (e != cudaSuccess) return cuda_fail("MLP parameter upload", e);
        const int smem = static_cast<int>(sizeof(MlpSmem));
        static const cudaError_t attr = cudaFuncSetAttribute(
            k_mlp_grad<true, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (attr != cudaSuccess) return cuda_fail("MLP kernel attribute", attr);
        const uint32_t blocks = (o->batch + kMlpBlock - 1) / kMlpBlock;
        for (uint32_t st = 0; st < o->steps; ++st) {
            if (st + 1 == o->steps) {
                e = cudaMemsetAsync(loss, 0, sizeof(float), s);
                if (e != cudaSuccess) return cuda_fail("loss reset", e);
            }
            k_mlp_grad<true, K><<<blocks, kMlpBlock, smem, s>>>(p, nullptr, nullptr, o->batch, t, md, o->seed, st, g,
                                                                loss);
            k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(p, g, m1, m2, st, o->lr);
        }
        e = cudaMemcpyAsync(&mdl->info.final_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail("loss read", e);
    }
    uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(mdl->d_mem));
    e = cudaMemsetAsync(err, 0, 256 + kErrRanges * sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail("error word reset", e);
    k_model_err<K><<<grid, 256, 0, s>>>(t, md, err, const_cast<uint32_t *>(md.errs));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("model kernels launch", e);
    uint32_t h_err = 0;
    e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail("model training", e);
    md.err = h_err;
    mdl->info.max_err = h_err;
    (void)n;
    (void)L;
    return BT_OK;
}

}  // namespace btgb

using namespace btgb;

extern "C" bt_status bt_model_train(const bt_tree *tree, const bt_learn_opts *opts, bt_stream stream,
                                    bt_model **out)
{
    if (!tree || !opts || !out) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    if (t.height == 0 || t.key_bytes == 32) return BT_ERR_ARG;
    if (opts->kind != BT_MODEL_PL && opts->kind != BT_MODEL_MLP) return BT_ERR_ARG;
    const uint64_t n = tree->info.n;
    const uint64_t L = t.nodes[t.height - 1];
    uint32_t S = 0;
    if (opts->kind == BT_MODEL_PL) {
        if (opts->segments == 0 || opts->segments > 65536) return BT_ERR_ARG;
        S = opts->segments < n ? opts->segments : static_cast<uint32_t>(n);
    } else {
        if (!opts->h_init || opts->steps == 0 || opts->batch == 0 || opts->batch > (1u << 22) ||
            !(opts->lr > 0.0f))
            return BT_ERR_ARG;
    }
    bt_model *m = new (std::nothrow) bt_model;
    if (!m) return BT_ERR_NOMEM;
    memset(m, 0, sizeof(*m));
    // device memory: err word | leaf_max | model arrays
    const uint64_t kb = t.key_bytes;
    uint64_t off = 256 + kErrRanges * 4;  // err word, then the per-range bounds
    const uint64_t off_lmax = off;
    off = a256(off + L * kb);
    uint64_t off_b = 0, off_inv = 0, off_slope = 0, off_icpt = 0, off_mlp = 0;
    if (opts->kind == BT_MODEL_PL) {
        off_b = off;
        off = a256(off + S * 8ull);
        off_inv = off;
        off = a256(off + S * 4ull);
        off_slope = off;
        off = a256(off + S * 4ull);
        off_icpt = off;
        off = a256(off + S * 4ull);
        off = a256(off + S * 5ull * 8ull + 256);  // fit sums (aligned after icpt)
    } else {
        off_b = off;
        off = a256(off + kMlpStage1 * 8ull);
        off_inv = off;
        off = a256(off + kMlpStage1 * 4ull);
        off_mlp = off;
        off = a256(off + (4ull * kMlpParams + 1) * 4ull);
    }
    cudaError_t e = cudaMalloc(&m->d_mem, off);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail("cudaMalloc(model)", e);
    }
    unsigned char *base = static_cast<unsigned char *>(m->d_mem);
    ModelDev &md = m->dev;
    md.kind = opts->kind;
    md.segments = S;
    md.leaves = static_cast<uint32_t>(L);
    md.leaf_max = base + off_lmax;
    md.errs = reinterpret_cast<const uint32_t *>(base + 256);
    md.kmin = t.kmin;
    md.kmax = t.kmax;
    md.inv_range = (t.kmax > t.kmin) ? static_cast<float>(1.0 / static_cast<double>(t.kmax - t.kmin)) : 0.0f;
    if (opts->kind == BT_MODEL_PL) {
        md.b = reinterpret_cast<const uint64_t *>(base + off_b);
        md.inv_w = reinterpret_cast<const float *>(base + off_inv);
        md.slope = reinterpret_cast<const float *>(base + off_slope);
        md.icpt = reinterpret_cast<const float *>(base + off_icpt);
    } else {
        md.b = reinterpret_cast<const uint64_t *>(base + off_b);
        md.inv_w = reinterpret_cast<const float *>(base + off_inv);
        md.mlp = reinterpret_cast<const float *>(base + off_mlp);
    }
    m->info.kind = opts->kind;
    m->info.segments = S;
    m->info.leaves = static_cast<uint32_t>(L);
    m->info.device_bytes = off;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bt_status st = (t.key_bytes == 8) ? train_impl<uint64_t>(tree, opts, s, m)
                                            : train_impl<uint32_t>(tree, opts, s, m);
    if (st != BT_OK) {
        cudaFree(m->d_mem);
        delete m;
        return st;
    }
    *out = m;
    return BT_OK;
}

extern "C" void bt_model_free(bt_model *m)
{
    if (!m) return;
    if (m->d_mem) cudaFree(m->d_mem);
    delete m;
}

extern "C" bt_status bt_model_get_info(const bt_model *m, bt_model_info *out)
{
    if (!m || !out) return BT_ERR_ARG;
    *out = m->info;
    return BT_OK;
}

extern "C" bt_status bt_model_copy_params(const bt_model *m, void *h_dst, uint64_t bytes)
{
    if (!m || !h_dst) return BT_ERR_ARG;
    const ModelDev &md = m->dev;
    cudaError_t e = cudaSuccess;
    unsigned char *d = static_cast<unsigned char *>(h_dst);
    if (md.kind == kModelPL) {
        const uint64_t S = md.segments;
        if (bytes < S * 20) return BT_ERR_ARG;
        e = cudaMemcpy(d, md.b, S * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(d + S * 8, md.inv_w, S * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(d + S * 12, md.slope, S * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(d + S * 16, md.icpt, S * 4, cudaMemcpyDeviceToHost);
    } else {
        if (bytes < kMlpParams * 4ull) return BT_ERR_ARG;
        e = cudaMemcpy(d, md.mlp, kMlpParams * 4ull, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail("model parameter copy", e);
    return BT_OK;
}

extern "C" bt_status bt_model_copy_err_bounds(const bt_model *m, uint32_t *h_dst, uint32_t n)
{
    if (!m || !h_dst || n < kErrRanges) return BT_ERR_ARG;
    const cudaError_t e = cudaMemcpy(h_dst, m->dev.errs, kErrRanges * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("error bound copy", e);
    return BT_OK;
}

extern "C" bt_status bt_mlp_grad(const float *d_params, const float *d_x, const float *d_t, uint32_t n,
                                 float *d_grad, float *d_loss, bt_stream stream)
{
    if (!d_params || !d_grad || !d_loss || (n && (!d_x || !d_t))) return BT_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_grad, 0, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail("gradient reset", e);
    if (n == 0) return BT_OK;
    const int smem = static_cast<int>(sizeof(MlpSmem));
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_mlp_grad<false, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return cuda_fail("MLP kernel attribute", attr);
    DevTree none;
    memset(&none, 0, sizeof(none));
    ModelDev md;
    memset(&md, 0, sizeof(md));
    k_mlp_grad<false, uint64_t><<<(n + kMlpBlock - 1) / kMlpBlock, kMlpBlock, smem, s>>>(
        d_params, d_x, d_t, n, none, md, 0, 0, d_grad, d_loss);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("MLP gradient launch", e);
    return BT_OK;
}
