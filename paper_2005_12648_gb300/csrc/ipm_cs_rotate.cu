// Circular shifting (Sec. 3.4) on the GPU: the exchange [X | Y] -> [Y | X] by cycle
// following, every element read once and written once.
//
// With n = |X| + |Y|, position x receives the element at (x + |X|) mod n, so the
// positions fall into g = gcd(|X|, n) cycles x_0 = c, x_{k+1} = (x_k + |X|) mod n of
// L = n / g positions each (c = 0 .. g-1); the exchange is p[x_k] <- p[x_{k+1}] along
// every cycle, the last position taking the cycle's first value.  The paper follows
// each cycle with one thread.  Here a cycle longer than the per-worker share S is cut
// into segments of S steps, each a worker of its own: a first launch saves every
// segment's first value (the value the previous segment's last step needs), a second
// runs all segments at once.  Workers are numbered cycle-fastest, so the lanes of a
// warp walk 32 neighbouring cycles in step and their accesses coalesce when g >= 32;
// with few cycles the lanes walk far-apart segments of one cycle and every access is a
// separate memory sector, several times slower than the tiled one-pass exchange of LS.
// This is the GPU side of the paper's open question whether CS can beat LS: only when
// the exchange has many cycles.
#include "ipm_internal.h"

namespace ipm {
namespace {

constexpr uint64_t kCsWorkers = 1ull << 18;  // target number of concurrent workers
constexpr uint64_t kCsMinSteps = 32;          // smallest per-worker share
constexpr int kCsUnroll = 8;                  // loads in flight per worker

// x_k of cycle c: (c + k |X|) mod n.
__device__ __forceinline__ uint64_t cs_pos(uint64_t c, uint64_t k, uint64_t lx, uint64_t n) {
    const uint64_t off = uint64_t((unsigned __int128)k * lx % n);
    const uint64_t x = c + off;
    return x >= n ? x - n : x;
}

template <typename T>
__global__ void cs_save_kernel(const T *__restrict__ p, uint64_t n, uint64_t lx, uint64_t g,
                               uint64_t S, uint64_t W, T *__restrict__ save) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < W; w += stride) {
        const uint64_t c = w % g, s = w / g;
        save[w] = p[cs_pos(c, s * S, lx, n)];
    }
}

// Segmented mode: worker w is cycle c = w mod g, steps [k0, k1) with k0 = (w / g) S.
template <typename T>
__global__ void cs_shift_kernel(T *p, uint64_t n, uint64_t lx, uint64_t g, uint64_t L,
                                uint64_t S, uint64_t nw, const T *__restrict__ save) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < nw; w += stride) {
        const uint64_t c = w % g;
        const uint64_t k0 = (w / g) * S;
        const uint64_t k1 = k0 + S < L ? k0 + S : L;
        uint64_t x = cs_pos(c, k0, lx, n);
        uint64_t k = k0;
        // p[x_k] <- p[x_{k+1}] for k in [k0, k1 - 1): kCsUnroll loads, then their stores
        // (every load of a batch is of a position this worker has not written yet)
        while (k + kCsUnroll < k1) {
            uint64_t y[kCsUnroll];
            T v[kCsUnroll];
            uint64_t q = x;
#pragma unroll
            for (int j = 0; j < kCsUnroll; ++j) {
                q += lx;
                q = q >= n ? q - n : q;
                y[j] = q;
            }
#pragma unroll
            for (int j = 0; j < kCsUnroll; ++j) v[j] = p[y[j]];
            p[x] = v[0];
#pragma unroll
            for (int j = 1; j < kCsUnroll; ++j) p[y[j - 1]] = v[j];
            x = y[kCsUnroll - 1];
            k += kCsUnroll;
        }
        while (k + 1 < k1) {
            uint64_t q = x + lx;
            q = q >= n ? q - n : q;
            p[x] = p[q];
            x = q;
            ++k;
        }
        // x = x_{k1-1} takes x_{k1}: the next segment's saved first value (segment 0 of
        // the same cycle after the last segment)
        p[x] = save[k1 == L ? c : w + g];
    }
}

// Whole-cycle mode (every cycle at most S steps): each thread follows kCsUnroll cycles
// c, c + stride, ... in step, keeping each cycle's first value in a register.
template <typename T>
__global__ void cs_whole_kernel(T *p, uint64_t n, uint64_t lx, uint64_t g, uint64_t L) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < g;
         base += stride * kCsUnroll) {
        uint64_t x[kCsUnroll];
        T first[kCsUnroll];
#pragma unroll
        for (int j = 0; j < kCsUnroll; ++j) {
            x[j] = base + uint64_t(j) * stride;  // the cycle's start, x_0 = c
            if (x[j] < g) first[j] = p[x[j]];
        }
        for (uint64_t k = 0; k + 1 < L; ++k) {
            T v[kCsUnroll];
            uint64_t y[kCsUnroll];
#pragma unroll
            for (int j = 0; j < kCsUnroll; ++j) {
                const uint64_t q = x[j] + lx;
                y[j] = q >= n ? q - n : q;
                if (base + uint64_t(j) * stride < g) v[j] = p[y[j]];
            }
#pragma unroll
            for (int j = 0; j < kCsUnroll; ++j) {
                if (base + uint64_t(j) * stride < g) p[x[j]] = v[j];
                x[j] = y[j];
            }
        }
#pragma unroll
        for (int j = 0; j < kCsUnroll; ++j)
            if (base + uint64_t(j) * stride < g) p[x[j]] = first[j];
    }
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b != 0) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

template <typename T>
ipm_status cs_rotate_t(void *ptr, const CsPlan &pl, void *save, cudaStream_t stream) {
    T *p = static_cast<T *>(ptr);
    const int threads = 256;
    const uint64_t cap = uint64_t(num_sms()) * 8;  // blocks: 8 x 256 threads per SM
    const uint64_t nw = pl.whole ? pl.g : pl.W;
    const uint64_t want = (nw + threads - 1) / threads;
    const unsigned blocks = unsigned(want < cap ? want : cap);
    if (pl.whole) {
        cs_whole_kernel<T><<<blocks, threads, 0, stream>>>(p, pl.n, pl.lx, pl.g, pl.L);
        return last_launch_status();
    }
    T *sv = static_cast<T *>(save);
    cs_save_kernel<T><<<blocks, threads, 0, stream>>>(p, pl.n, pl.lx, pl.g, pl.S, pl.W, sv);
    IPM_TRY(last_launch_status());
    cs_shift_kernel<T><<<blocks, threads, 0, stream>>>(p, pl.n, pl.lx, pl.g, pl.L, pl.S,
                                                       nw, sv);
    return last_launch_status();
}

}  // namespace

CsPlan cs_plan(uint64_t lx, uint64_t ly) {
    CsPlan pl{};
    pl.lx = lx;
    pl.n = lx + ly;
    if (lx == 0 || ly == 0) return pl;
    pl.g = gcd_u64(lx, ly);  // = gcd(lx, n)
    pl.L = pl.n / pl.g;
    const uint64_t share = (pl.n + kCsWorkers - 1) / kCsWorkers;
    pl.S = share > kCsMinSteps ? share : kCsMinSteps;
    pl.whole = pl.L <= pl.S;
    // segments: W = g ceil(L / S) < n / S + g <= 2 kCsWorkers (L > S implies g < n / S)
    pl.W = pl.whole ? 0 : pl.g * ((pl.L + pl.S - 1) / pl.S);
    return pl;
}

ipm_status launch_cs_rotate(void *ptr, uint32_t elem_bytes, const CsPlan &pl, void *save,
                            cudaStream_t stream) {
    if (pl.g == 0) return IPM_OK;
    return elem_bytes == 4 ? cs_rotate_t<uint32_t>(ptr, pl, save, stream)
                           : cs_rotate_t<uint64_t>(ptr, pl, save, stream);
}

}  // namespace ipm
