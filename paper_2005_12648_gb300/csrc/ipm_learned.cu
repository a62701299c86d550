// Learned split proposer (no counterpart in the paper; it extends the split step of
// Sec. 3.1): a 1 -> 32 -> 1 tanh MLP in FP32 predicts the split of a diagonal from its
// relative position, a warp corrects the proposal to the exact split.
//
//   model      y(x) = b2 + sum_h w2[h] tanh(w1[h] x + b1[h]), x = d / n, target i / len_a.
//              One warp evaluates it with lane h holding hidden unit h (32 = warp size).
//   training   targets: the exact split of every sample diagonal (warp_split); then
//              full-batch Adam on the mean squared error, all steps in one CTA: each warp
//              takes a share of the samples and accumulates the gradient of its lane's
//              hidden unit, the warps' partial sums are added in shared memory, and
//              threads 0..96 apply the Adam update to the parameters held there.
//   correction one round of 32 probes at exponentially spaced offsets around the
//              proposal (galloping: -2^15 .. -1, 0, 1, 3, ..., 2^15-1, clamped to the
//              diagonal's range) brackets the split; the bracket search of the plain
//              split finishes it.  The result is the exact split whatever the proposal.
#include "ipm_internal.h"
#include "ipm_split.cuh"

namespace ipm {

namespace {

constexpr int kH = IPM_SPLIT_MODEL_HIDDEN;
constexpr int kNP = 3 * kH + 1;           // parameters: w1, b1, w2, b2
constexpr int kTrainThreads = 1024;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr uint32_t kMaxSamples = 1u << 20;
static_assert(kH == 32, "one hidden unit per lane");

// Parameter q of a model held as the ipm_split_model layout (w1 | b1 | w2 | b2).
__device__ __forceinline__ const float *model_params(const ipm_split_model *m) {
    return m->w1;
}

// y(x) by one warp: lane h adds w2[h] tanh(w1[h] x + b1[h]); the butterfly leaves the
// same sum in every lane.
__device__ __forceinline__ float warp_mlp(const float *prm, float x) {
    const unsigned h = threadIdx.x & 31u;
    float u = prm[2 * kH + h] * tanhf(fmaf(prm[h], x, prm[kH + h]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    return prm[3 * kH] + u;
}

// Mean squared error and its gradient over the n samples, by the whole CTA; prm is in
// shared memory.  red holds kTrainWarps x (kNP + 1) partial sums; on return out[0..96]
// holds the gradient (w1, b1, w2, b2) and out[97] the loss.
__device__ void block_loss_grad(const float *prm, const float *xs, const float *ts, uint32_t n,
                                float (*red)[kNP + 1], float *out) {
    const uint32_t tid = threadIdx.x, warp = tid >> 5, h = tid & 31u;
    const float w1 = prm[h], b1 = prm[kH + h], w2 = prm[2 * kH + h], b2 = prm[3 * kH];
    const float two_over_n = 2.0f / float(n);
    float gw1 = 0.f, gb1 = 0.f, gw2 = 0.f, gb2 = 0.f, loss = 0.f;
    for (uint32_t s = warp; s < n; s += kTrainWarps) {
        const float x = xs[s], t = ts[s];
        const float a = tanhf(fmaf(w1, x, b1));
        float u = w2 * a;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        const float r = (b2 + u) - t;
        const float g = two_over_n * r;             // dL/dy
        const float du = g * w2 * (1.0f - a * a);   // dL/du, u = w1 x + b1
        gw1 = fmaf(du, x, gw1);
        gb1 += du;
        gw2 = fmaf(g, a, gw2);
        gb2 += g;
        loss = fmaf(r, r, loss);
    }
    red[warp][h] = gw1;
    red[warp][kH + h] = gb1;
    red[warp][2 * kH + h] = gw2;
    if (h == 0) {
        red[warp][3 * kH] = gb2;
        red[warp][kNP] = loss;
    }
    __syncthreads();
    if (tid <= uint32_t(kNP)) {
        float sum = 0.f;
        for (int w = 0; w < kTrainWarps; ++w) sum += red[w][tid];
        out[tid] = tid == uint32_t(kNP) ? sum / float(n) : sum;
    }
    __syncthreads();
}

// Samples staged in shared memory up to this count (x and t: 8 bytes each; the static
// shared memory of the training kernel stays under 48 KiB).
constexpr uint32_t kSmemSamples = 4096;

__global__ void __launch_bounds__(kTrainThreads, 1)
    train_kernel(const float *__restrict__ gx, const float *__restrict__ gt, uint32_t n,
                 ipm_split_train_options opt, ipm_split_model *model) {
    __shared__ float prm[kNP], mom1[kNP], mom2[kNP], grad[kNP + 1];
    __shared__ float red[kTrainWarps][kNP + 1];
    __shared__ float sx[kSmemSamples], st[kSmemSamples];
    const uint32_t tid = threadIdx.x;
    const float *mp = model_params(model);
    if (tid < uint32_t(kNP)) {
        prm[tid] = mp[tid];
        mom1[tid] = 0.f;
        mom2[tid] = 0.f;
    }
    const bool staged = n <= kSmemSamples;
    if (staged)
        for (uint32_t s = tid; s < n; s += kTrainThreads) {
            sx[s] = gx[s];
            st[s] = gt[s];
        }
    __syncthreads();
    const float *xs = staged ? sx : gx;
    const float *ts = staged ? st : gt;
    float b1t = 1.f, b2t = 1.f;  // beta1^step, beta2^step
    for (uint32_t step = 1; step <= opt.steps; ++step) {
        block_loss_grad(prm, xs, ts, n, red, grad);
        b1t *= opt.beta1;
        b2t *= opt.beta2;
        if (tid < uint32_t(kNP)) {
            const float g = grad[tid];
            const float m = opt.beta1 * mom1[tid] + (1.f - opt.beta1) * g;
            const float v = opt.beta2 * mom2[tid] + (1.f - opt.beta2) * g * g;
            mom1[tid] = m;
            mom2[tid] = v;
            prm[tid] -= opt.lr * (m / (1.f - b1t)) / (sqrtf(v / (1.f - b2t)) + opt.eps);
        }
        __syncthreads();
    }
    block_loss_grad(prm, xs, ts, n, red, grad);  // loss of the trained parameters
    float *out = model->w1;
    if (tid < uint32_t(kNP)) out[tid] = prm[tid];
    if (tid == 0) {
        model->loss = grad[kNP];
        model->steps = opt.steps;
    }
}

__global__ void __launch_bounds__(kTrainThreads, 1)
    loss_grad_kernel(const ipm_split_model *model, const float *__restrict__ x,
                     const float *__restrict__ t, uint32_t n, float *out) {
    __shared__ float prm[kNP], grad[kNP + 1];
    __shared__ float red[kTrainWarps][kNP + 1];
    const uint32_t tid = threadIdx.x;
    if (tid < uint32_t(kNP)) prm[tid] = model_params(model)[tid];
    __syncthreads();
    block_loss_grad(prm, x, t, n, red, grad);
    if (tid <= uint32_t(kNP)) out[tid] = grad[tid];
}

__global__ void __launch_bounds__(256)
    forward_kernel(const ipm_split_model *model, const float *__restrict__ x, uint32_t n,
                   float *y) {
    __shared__ float prm[kNP];
    if (threadIdx.x < uint32_t(kNP)) prm[threadIdx.x] = model_params(model)[threadIdx.x];
    __syncthreads();
    const uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n) return;  // whole warp
    const float v = warp_mlp(prm, x[s]);
    if ((threadIdx.x & 31u) == 0) y[s] = v;
}

// Training targets: x_s = d_s / n, t_s = i_s / len_a with i_s the exact split of d_s.
template <typename K>
__global__ void __launch_bounds__(256)
    targets_kernel(const K *__restrict__ A, uint64_t la, const K *__restrict__ B, uint64_t lb,
                   const uint64_t *__restrict__ diags, uint32_t n, float *x, float *t,
                   StatusBlock *sb) {
    const uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n) return;  // whole warp
    const uint64_t total = la + lb;
    uint64_t d = diags[s];
    if (d > total) {
        if ((threadIdx.x & 31u) == 0) set_status(sb, IPM_ERR_INVALID_ARG);
        d = total;
    }
    const uint64_t i = warp_split<true>(A, la, B, lb, d);
    if ((threadIdx.x & 31u) == 0) {
        x[s] = float(double(d) / double(total));
        t[s] = float(double(i) / double(la));
    }
}

__global__ void reset_status_kernel(StatusBlock *sb) {
    if (threadIdx.x == 0) sb->status = 0u;
}

// Accumulate one diagonal's search counts and proposal error (lane 0).
__device__ __forceinline__ void add_stats(ipm_split_stats *stats, uint32_t rounds,
                                          uint32_t probes, uint64_t err) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&stats->diagonals), 1ull);
    atomicAdd(reinterpret_cast<unsigned long long *>(&stats->rounds),
              (unsigned long long)rounds);
    atomicAdd(reinterpret_cast<unsigned long long *>(&stats->probes),
              (unsigned long long)probes);
    atomicAdd(reinterpret_cast<unsigned long long *>(&stats->abs_err_sum),
              (unsigned long long)err);
    atomicMax(reinterpret_cast<unsigned long long *>(&stats->abs_err_max),
              (unsigned long long)err);
}

// One galloping round from `guess` inside [lo, hi): the lanes probe the offsets
// -2^15 .. -1 (lanes 0..15), 0, 1, 3, .., 2^15 - 1 around it (clamped to the range) at
// once, and the ballot narrows [lo, hi] to the bracket that holds the split.
template <typename K>
__device__ __forceinline__ void gallop_round(const K *A, const K *B, uint64_t d, uint64_t guess,
                                             uint64_t &lo, uint64_t &hi) {
    const unsigned lane = threadIdx.x & 31u;
    const int64_t off = lane < 16 ? -(int64_t(1) << (15 - lane)) : (int64_t(1) << (lane - 16)) - 1;
    int64_t m = int64_t(guess) + off;
    const int64_t mlo = int64_t(lo), mhi = int64_t(hi) - 1;
    m = m < mlo ? mlo : m > mhi ? mhi : m;
    const bool p = key_le(A[m], B[d - 1 - uint64_t(m)]);
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    const int64_t m_lo = __shfl_sync(0xffffffffu, m, c > 0 ? c - 1 : 0);
    const int64_t m_hi = __shfl_sync(0xffffffffu, m, c < 32 ? c : 31);
    if (c > 0) lo = uint64_t(m_lo) + 1;
    if (c < 32) hi = uint64_t(m_hi);
}

// Exact splits on d_k = floor(k*n/P) for k = 0, S, 2S, ..., P (S = stride) from the
// model's proposals (MODEL) or by the plain bracket search; STATS accumulates probe
// counts and proposal errors.
template <typename K, bool MODEL, bool STATS>
__global__ void __launch_bounds__(256)
    learned_split_kernel(const K *__restrict__ A, uint64_t la, const K *__restrict__ B,
                         uint64_t lb, uint64_t P, uint64_t stride, const ipm_split_model *model,
                         uint64_t *__restrict__ out, ipm_split_stats *stats,
                         const StatusBlock *sb) {
    __shared__ float prm[kNP];
    if (MODEL) {
        if (threadIdx.x < uint32_t(kNP)) prm[threadIdx.x] = model_params(model)[threadIdx.x];
        __syncthreads();
    }
    if (call_finished(sb)) return;
    const uint64_t k = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * stride;
    const unsigned lane = threadIdx.x & 31u;
    if (k > P) return;  // whole warp exits together
    const uint64_t n = la + lb;
    const uint64_t d = (k * n) / P;
    uint64_t lo = d > lb ? d - lb : 0;
    uint64_t hi = d < la ? d : la;
    uint64_t guess = lo;
    uint32_t rounds = 0, probes = 0;
    if (MODEL && hi > lo) {
        const float y = warp_mlp(prm, float(double(d) / double(n)));
        const double g = rint(double(y) * double(la));
        // clamp to the diagonal's range (a NaN proposal becomes lo)
        guess = g > double(lo) ? (g < double(hi) ? uint64_t(g) : hi) : lo;
        gallop_round(A, B, d, guess, lo, hi);
        rounds = 1;
        probes = 32;
    }
    uint32_t r2 = 0, p2 = 0;
    const uint64_t i = warp_split_bracket<true, STATS>(A, B, d, lo, hi, &r2, &p2);
    if (lane == 0) {
        out[k] = i;
        if (STATS) add_stats(stats, rounds + r2, probes + p2,
                             MODEL ? (guess > i ? guess - i : i - guess) : 0);
    }
}

// The other diagonals, once those of learned_split_kernel with this stride are known:
// the split lies in the bracket of its coarse neighbours k0 < k < k1 (both i_k and
// j_k = d_k - i_k grow with k).  With PROPOSE the search starts at the piecewise-linear
// model through the exact coarse splits (i_k0 + (i_k1 - i_k0) (d_k - d_k0) / (d_k1 -
// d_k0), clamped to the bracket) with one galloping round; without, the plain bracket
// search.
template <typename K, bool PROPOSE, bool STATS>
__global__ void __launch_bounds__(256)
    learned_fine_kernel(const K *__restrict__ A, uint64_t la, const K *__restrict__ B,
                        uint64_t lb, uint64_t P, uint64_t stride, uint64_t *__restrict__ out,
                        ipm_split_stats *stats, const StatusBlock *sb) {
    if (call_finished(sb)) return;
    const uint64_t k = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (k > P || k % stride == 0) return;  // whole warp exits together
    const uint64_t n = la + lb;
    const uint64_t k0 = k / stride * stride, k1 = k0 + stride;  // k1 <= P: stride | P
    const uint64_t d = (k * n) / P, d0 = (k0 * n) / P, d1 = (k1 * n) / P;
    const uint64_t i0 = out[k0], i1 = out[k1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    uint64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    if (i0 > lo) lo = i0;
    if (d > j1 && d - j1 > lo) lo = d - j1;
    if (i1 < hi) hi = i1;
    if (d - j0 < hi) hi = d - j0;
    uint64_t guess = lo;
    uint32_t rounds = 0, probes = 0;
    if (PROPOSE && hi > lo) {
        const double g = double(i0) + rint(double(i1 - i0) * (double(d - d0) / double(d1 - d0)));
        guess = g > double(lo) ? (g < double(hi) ? uint64_t(g) : hi) : lo;
        gallop_round(A, B, d, guess, lo, hi);
        rounds = 1;
        probes = 32;
    }
    uint32_t r2 = 0, p2 = 0;
    const uint64_t i = warp_split_bracket<true, STATS>(A, B, d, lo, hi, &r2, &p2);
    if (lane == 0) {
        out[k] = i;
        if (STATS) add_stats(stats, rounds + r2, probes + p2,
                             PROPOSE ? (guess > i ? guess - i : i - guess) : 0);
    }
}

// Every 32nd diagonal first when there are 2,048 or more (a multiple of 32), then the
// others inside the brackets of their coarse neighbours; with a model, the coarse
// diagonals start at the model's proposals and the fine ones at the piecewise-linear
// model through the coarse splits.  Without a model, the plain searches of
// ipm_merge_splits.
constexpr uint64_t kLearnedStride = 32;
constexpr uint64_t kLearnedTwoPass = 2048;

template <typename K, bool MODEL, bool STATS>
ipm_status learned_splits_v(const K *A, uint64_t la, uint64_t lb, uint64_t P,
                            const ipm_split_model *model, uint64_t *split,
                            ipm_split_stats *stats, const StatusBlock *sb,
                            cudaStream_t stream) {
    const bool two = P >= kLearnedTwoPass && P % kLearnedStride == 0;
    const uint64_t stride = two ? kLearnedStride : 1;
    const uint64_t blocks = ((P / stride + 1) * 32 + 255) / 256;
    const uint64_t fblocks = ((P + 1) * 32 + 255) / 256;
    if (fblocks > 0x7fffffffull) return IPM_ERR_INVALID_ARG;
    learned_split_kernel<K, MODEL, STATS><<<unsigned(blocks), 256, 0, stream>>>(
        A, la, A + la, lb, P, stride, model, split, stats, sb);
    if (!two) return last_launch_status();
    IPM_TRY(last_launch_status());
    learned_fine_kernel<K, MODEL, STATS><<<unsigned(fblocks), 256, 0, stream>>>(
        A, la, A + la, lb, P, stride, split, stats, sb);
    return last_launch_status();
}

template <typename K>
ipm_status learned_splits_t(const void *buf, uint64_t la, uint64_t lb, uint64_t P,
                            const ipm_split_model *model, uint64_t *split,
                            ipm_split_stats *stats, const StatusBlock *sb,
                            cudaStream_t stream) {
    const K *A = static_cast<const K *>(buf);
    if (model != nullptr)
        return stats != nullptr
                   ? learned_splits_v<K, true, true>(A, la, lb, P, model, split, stats, sb, stream)
                   : learned_splits_v<K, true, false>(A, la, lb, P, model, split, nullptr, sb,
                                                      stream);
    return stats != nullptr
               ? learned_splits_v<K, false, true>(A, la, lb, P, nullptr, split, stats, sb, stream)
               : learned_splits_v<K, false, false>(A, la, lb, P, nullptr, split, nullptr, sb,
                                                   stream);
}

template <typename K>
ipm_status targets_t(const void *buf, uint64_t la, uint64_t lb, const uint64_t *diags,
                     uint32_t n, float *x, float *t, StatusBlock *sb, cudaStream_t stream) {
    const K *A = static_cast<const K *>(buf);
    const unsigned blocks = unsigned((uint64_t(n) * 32 + 255) / 256);
    targets_kernel<K><<<blocks, 256, 0, stream>>>(A, la, A + la, lb, diags, n, x, t, sb);
    return last_launch_status();
}

}  // namespace

uint32_t learned_split_launches(uint64_t P) {
    return P >= kLearnedTwoPass && P % kLearnedStride == 0 ? 2u : 1u;
}

ipm_status launch_learned_splits(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                                 uint64_t P, const ipm_split_model *model, uint64_t *split,
                                 ipm_split_stats *stats, const StatusBlock *sb,
                                 cudaStream_t stream) {
    switch (key) {
    case IPM_INT32:
        return learned_splits_t<int32_t>(buf, la, lb, P, model, split, stats, sb, stream);
    case IPM_UINT32:
        return learned_splits_t<uint32_t>(buf, la, lb, P, model, split, stats, sb, stream);
    case IPM_UINT64:
        return learned_splits_t<uint64_t>(buf, la, lb, P, model, split, stats, sb, stream);
    case IPM_INT64:
        return learned_splits_t<int64_t>(buf, la, lb, P, model, split, stats, sb, stream);
    case IPM_FLOAT32:
        return learned_splits_t<float>(buf, la, lb, P, model, split, stats, sb, stream);
    }
    return IPM_ERR_UNSUPPORTED_DTYPE;
}

size_t split_model_train_ws_bytes(uint32_t nsamples) {
    return kStatusBytes + align_up(sizeof(float) * size_t(nsamples), 256) * 2;
}

ipm_status launch_split_model_train(const void *buf, uint64_t la, uint64_t lb, ipm_dtype key,
                                    const uint64_t *diags, uint32_t n,
                                    const ipm_split_train_options &opt,
                                    ipm_split_model *model, void *ws, cudaStream_t stream) {
    if (n == 0 || n > kMaxSamples) return IPM_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    StatusBlock *sb = reinterpret_cast<StatusBlock *>(w);
    float *x = reinterpret_cast<float *>(w + kStatusBytes);
    float *t = reinterpret_cast<float *>(w + kStatusBytes +
                                         align_up(sizeof(float) * size_t(n), 256));
    reset_status_kernel<<<1, 32, 0, stream>>>(sb);
    IPM_TRY(last_launch_status());
    switch (key) {
    case IPM_INT32:
        IPM_TRY(targets_t<int32_t>(buf, la, lb, diags, n, x, t, sb, stream));
        break;
    case IPM_UINT32:
        IPM_TRY(targets_t<uint32_t>(buf, la, lb, diags, n, x, t, sb, stream));
        break;
    case IPM_UINT64:
        IPM_TRY(targets_t<uint64_t>(buf, la, lb, diags, n, x, t, sb, stream));
        break;
    case IPM_INT64:
        IPM_TRY(targets_t<int64_t>(buf, la, lb, diags, n, x, t, sb, stream));
        break;
    case IPM_FLOAT32:
        IPM_TRY(targets_t<float>(buf, la, lb, diags, n, x, t, sb, stream));
        break;
    default:
        return IPM_ERR_UNSUPPORTED_DTYPE;
    }
    train_kernel<<<1, kTrainThreads, 0, stream>>>(x, t, n, opt, model);
    return last_launch_status();
}

ipm_status launch_split_model_forward(const ipm_split_model *model, const float *x, uint32_t n,
                                      float *y, cudaStream_t stream) {
    if (n == 0) return IPM_OK;
    const unsigned blocks = unsigned((uint64_t(n) * 32 + 255) / 256);
    forward_kernel<<<blocks, 256, 0, stream>>>(model, x, n, y);
    return last_launch_status();
}

ipm_status launch_split_model_loss_grad(const ipm_split_model *model, const float *x,
                                        const float *t, uint32_t n, float *grad,
                                        cudaStream_t stream) {
    if (n == 0 || n > kMaxSamples) return IPM_ERR_INVALID_ARG;
    loss_grad_kernel<<<1, kTrainThreads, 0, stream>>>(model, x, t, n, grad);
    return last_launch_status();
}

}  // namespace ipm
