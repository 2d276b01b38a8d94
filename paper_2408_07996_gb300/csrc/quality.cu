// quality.cu -- event-video quality metrics (Sec. 4.2): the frame error of
// the mapped event frames, and the distance from every event to the nearest
// event of the same polarity in the other video, behind the polarity-aware
// F1 score and chamfer distance.
//
// The distances are an exact squared Euclidean distance transform on the
// integer lattice (x, y, t), separable by axis:
//   rows (x): the input is binary, so a warp sweeps each row left to right
//     with a max-scan of event columns and right to left with a min-scan;
//   columns (y, then t): F'(u) = min_i (u - i)^2 + F(i) is the lower
//     envelope of parabolas rooted at the finite sites i of the line, built
//     in one forward sweep with integer separation points
//     floor((u^2 - i^2 + F(u) - F(i)) / (2 (u - i))) and read back in one
//     backward sweep (Meijster, Roerdink and Hesselink 2000; Felzenszwalb
//     and Huttenlocher 2012).  One thread owns one line at a time.  All
//     arithmetic is integer, so the result is exact.
#include <algorithm>
#include <climits>
#include <utility>

#include "quality.h"

namespace mcev {
namespace {

constexpr int32_t QINF = 1 << 30;
constexpr int QBLOCK = 256;
constexpr int SMEM_BUDGET = 220 * 1024;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sums of three counters and one double, one atomic per nonzero
// value per block (slots < 0 are skipped)
__device__ void block_flush(unsigned long long u0, unsigned long long u1, unsigned long long u2, double d0,
                            unsigned long long* acc, int s0, int s1, int s2, int sd) {
    __shared__ unsigned long long p0[QBLOCK / 32], p1[QBLOCK / 32], p2[QBLOCK / 32];
    __shared__ double pd[QBLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u0 = warp_sum(u0);
    u1 = warp_sum(u1);
    u2 = warp_sum(u2);
    d0 = warp_sum(d0);
    if (lane == 0) {
        p0[wid] = u0;
        p1[wid] = u1;
        p2[wid] = u2;
        pd[wid] = d0;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        u0 = warp_sum(lane < nw ? p0[lane] : 0ull);
        u1 = warp_sum(lane < nw ? p1[lane] : 0ull);
        u2 = warp_sum(lane < nw ? p2[lane] : 0ull);
        d0 = warp_sum(lane < nw ? pd[lane] : 0.0);
        if (lane == 0) {
            if (s0 >= 0 && u0) atomicAdd(acc + s0, u0);
            if (s1 >= 0 && u1) atomicAdd(acc + s1, u1);
            if (s2 >= 0 && u2) atomicAdd(acc + s2, u2);
            if (sd >= 0 && d0 != 0.0) atomicAdd(reinterpret_cast<double*>(acc + sd), d0);
        }
    }
}

// ---------------------------------------------------------------- frame error + counts
__device__ __forceinline__ void tally(int va, int vb, unsigned long long& sq, unsigned long long& na,
                                      unsigned long long& nb, unsigned& bad) {
    const int d = va - vb;
    sq += (unsigned long long)(d * d);
    na += va != 0;
    nb += vb != 0;
    bad |= (unsigned)(va < -1 || va > 1 || vb < -1 || vb > 1);
}

__global__ void __launch_bounds__(QBLOCK) k_frame_error(const int8_t* __restrict__ a, const int8_t* __restrict__ b,
                                                        int64_t n, int vec, unsigned long long* acc) {
    unsigned long long sq = 0, na = 0, nb = 0;
    unsigned bad = 0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const int64_t nv = n >> 4;
        const int4* a4 = reinterpret_cast<const int4*>(a);
        const int4* b4 = reinterpret_cast<const int4*>(b);
        for (int64_t i = tid; i < nv; i += nth) {
            const int4 x = __ldg(a4 + i), y = __ldg(b4 + i);
            const int xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int w = 0; w < 4; ++w)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tally((int)(int8_t)(xs[w] >> (8 * k)), (int)(int8_t)(ys[w] >> (8 * k)), sq, na, nb, bad);
        }
        done = nv << 4;
    }
    for (int64_t i = done + tid; i < n; i += nth) tally(a[i], b[i], sq, na, nb, bad);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(acc + QACC_BAD, 1ull);
    block_flush(sq, na, nb, 0.0, acc, QACC_SQ, QACC_NA, QACC_NB, -1);
}

// ---------------------------------------------------------------- rows: 1-D distance to the nearest event
// One warp per row; `left` (shared) keeps the column of the nearest event at
// or left of each x between the two sweeps.
__global__ void k_edt_rows(const int8_t* __restrict__ v, int W, int64_t rows, int pol, int32_t* __restrict__ out) {
    extern __shared__ int32_t q_left[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int32_t* left = q_left + (size_t)wib * W;
    for (int64_t r = (int64_t)blockIdx.x * wpb + wib; r < rows; r += (int64_t)gridDim.x * wpb) {
        const int8_t* src = v + r * W;
        int32_t* dst = out + r * W;
        int carry = -1;
        for (int x0 = 0; x0 < W; x0 += 32) {
            const int x = x0 + lane;
            int idx = (x < W && src[x] == pol) ? x : -1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, idx, o);
                if (lane >= o) idx = max(idx, y);
            }
            idx = max(idx, carry);
            if (x < W) left[x] = idx;
            carry = __shfl_sync(0xffffffffu, idx, 31);
        }
        carry = INT_MAX;
        for (int x0 = (W - 1) & ~31; x0 >= 0; x0 -= 32) {
            const int x = x0 + lane;
            int idx = (x < W && src[x] == pol) ? x : INT_MAX;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_down_sync(0xffffffffu, idx, o);
                if (lane + o < 32) idx = min(idx, y);
            }
            idx = min(idx, carry);
            if (x < W) {
                const int l = left[x];
                int32_t d = QINF;
                if (l >= 0) d = (x - l) * (x - l);
                if (idx != INT_MAX) d = min(d, (idx - x) * (idx - x));
                dst[x] = d;
            }
            carry = __shfl_sync(0xffffffffu, idx, 0);
        }
    }
}

// ---------------------------------------------------------------- columns: lower envelope of parabolas
constexpr int COL_PREFETCH = 16;

__device__ __forceinline__ int32_t floordiv32(int32_t a, int32_t b) {  // b > 0
    const int32_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// Line `line` = (outer, inner x): elements base + u * step, u = 0..L-1,
// base = outer * outer_stride + x.  The envelope is a stack of sites (site s,
// interval start t, site value f); its top lives in registers, the entries
// below it in global memory, entry (depth k, thread g) at k * G + g for the
// G threads of the launch, packed as (s | t << 16, f).  A thread owns one
// stack and walks lines g, g + G, ...; keeping the stacks out of shared
// memory lets every SM run at full occupancy, which hides the latency of the
// sweeps (stacks in shared memory held a 720-long line pass to 39 threads
// per SM and ran 6.7x slower).  The forward sweep loads 16 elements ahead.
// Every quantity fits in int32: extents <= 16384 keep squared distances
// <= 3 * 16383^2 < 2^30.
__global__ void __launch_bounds__(256) k_edt_cols(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                    int64_t n_lines, int W, int64_t outer_stride, int64_t step, int L,
                                                    int2* __restrict__ stack) {
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t line = g; line < n_lines; line += G) {
        const int64_t x = line % W, outer = line / W;
        const int32_t* src = in + outer * outer_stride + x;
        int32_t* dst = out + outer * outer_stride + x;
        int depth = 0;
        int32_t top_s = 0, top_t = 0, top_f = 0;
        for (int u0 = 0; u0 < L; u0 += COL_PREFETCH) {
            int32_t buf[COL_PREFETCH];
#pragma unroll
            for (int j = 0; j < COL_PREFETCH; ++j)
                buf[j] = u0 + j < L ? __ldg(src + (int64_t)(u0 + j) * step) : QINF;
#pragma unroll
            for (int j = 0; j < COL_PREFETCH; ++j) {
                const int32_t u = u0 + j, fu = buf[j];
                if (fu >= QINF) continue;
                while (depth > 0) {
                    const int32_t f_site = (top_t - top_s) * (top_t - top_s) + top_f;
                    const int32_t f_new = (top_t - u) * (top_t - u) + fu;
                    if (f_site <= f_new) break;
                    if (--depth > 0) {
                        const int2 e = stack[(int64_t)(depth - 1) * G + g];
                        top_s = e.x & 0xFFFF;
                        top_t = (int32_t)((uint32_t)e.x >> 16);
                        top_f = e.y;
                    }
                }
                if (depth == 0) {
                    depth = 1;
                    top_s = u;
                    top_t = 0;
                    top_f = fu;
                } else {
                    const int32_t w = 1 + floordiv32(u * u - top_s * top_s + fu - top_f, 2 * (u - top_s));
                    if (w < L) {
                        stack[(int64_t)(depth - 1) * G + g] = make_int2(top_s | (top_t << 16), top_f);
                        ++depth;
                        top_s = u;
                        top_t = w;
                        top_f = fu;
                    }
                }
            }
        }
        for (int32_t u = L - 1; u >= 0; --u) {
            int32_t d = QINF;
            if (depth > 0) {
                d = (u - top_s) * (u - top_s) + top_f;
                if (u == top_t && --depth > 0) {
                    const int2 e = stack[(int64_t)(depth - 1) * G + g];
                    top_s = e.x & 0xFFFF;
                    top_t = (int32_t)((uint32_t)e.x >> 16);
                    top_f = e.y;
                }
            }
            dst[(int64_t)u * step] = d;
        }
    }
}

// ---------------------------------------------------------------- matching of one polarity
__device__ __forceinline__ void match_one(int32_t d, int64_t i, int32_t* d2_out, int tau2, uint32_t* hist,
                                          unsigned long long& matched, unsigned long long& none, double& sum) {
    if (d >= QINF) {
        ++none;
        if (d2_out) d2_out[i] = -2;
    } else {
        matched += d <= tau2;
        if (d >= QHIST) sum += sqrt((double)d);
        else if (d > 0) atomicAdd(hist + d, 1u);
        if (d2_out) d2_out[i] = d;
    }
}

// vec: the query video is 4-byte aligned (the distance volume always is), so
// each thread takes 4 voxels per step with one 4-byte and one 16-byte load.
// Distances are tallied per squared value in a shared histogram.
__global__ void __launch_bounds__(QBLOCK) k_match(const int8_t* __restrict__ qv, const int32_t* __restrict__ d2,
                                                  int64_t n, int pol, int tau2, int vec, int32_t* __restrict__ d2_out,
                                                  unsigned long long* acc, int slot, unsigned long long* ghist) {
    __shared__ uint32_t hist[QHIST];
    for (int b = threadIdx.x; b < QHIST; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    unsigned long long matched = 0, none = 0;
    double sum = 0.0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = n >> 2;
        const int32_t* q4 = reinterpret_cast<const int32_t*>(qv);
        const int4* d4 = reinterpret_cast<const int4*>(d2);
        for (int64_t i = tid; i < n4; i += nth) {
            const int32_t qw = __ldg(q4 + i);
            if (qw == 0) continue;      // no event among the 4 voxels
            bool any = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) any |= (int)(int8_t)(qw >> (8 * k)) == pol;
            if (!any) continue;
            const int4 dv = __ldg(d4 + i);
            const int32_t ds[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((int)(int8_t)(qw >> (8 * k)) == pol)
                    match_one(ds[k], 4 * i + k, d2_out, tau2, hist, matched, none, sum);
        }
        done = n4 << 2;
    }
    for (int64_t i = done + tid; i < n; i += nth)
        if (qv[i] == pol) match_one(__ldg(d2 + i), i, d2_out, tau2, hist, matched, none, sum);
    block_flush(matched, none, 0ull, sum, acc, slot, slot + 1, -1, slot + 2);   // synchronises the block
    for (int b = threadIdx.x; b < QHIST; b += blockDim.x)
        if (hist[b]) atomicAdd(ghist + b, (unsigned long long)hist[b]);
}

// Blocks of 256 threads for the column kernel: enough for every line, at
// most 8 per SM, and no more than the stack scratch holds.
int stack_blocks(int64_t n_lines, int L, int sms) {
    const int64_t by_lines = (n_lines + 255) / 256;
    const int64_t by_sms = (int64_t)sms * 8;
    const int64_t by_mem = QUALITY_STACK_BYTES / (8 * (int64_t)L * 256);
    return (int)std::max<int64_t>(1, std::min(by_lines, std::min(by_sms, by_mem)));
}

int grid_of(int64_t work, int per_block, int sms, int per_sm) {
    const int64_t need = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sms * per_sm;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace

int64_t quality_stack_bytes(int32_t W, int32_t H, int32_t T, int sms) {
    const int64_t lines[2] = {(int64_t)T * W, (int64_t)H * W}, len[2] = {H, T};
    int64_t need = 0;
    for (int ax = 0; ax < 2; ++ax) {
        if (len[ax] < 2) continue;
        const int b = stack_blocks(lines[ax], (int)len[ax], sms);
        need = std::max<int64_t>(need, (int64_t)b * 256 * len[ax] * 8);
    }
    return need;
}

cudaError_t launch_quality(const QualityArgs& A, int sms, cudaStream_t st, int* launches) {
    static bool attrs[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attrs[dev]) {
        if ((e = cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BUDGET)) !=
            cudaSuccess)
            return e;
        if (dev >= 0 && dev < 64) attrs[dev] = true;
    }
    int nl = 0;
    const int64_t W = A.W, H = A.H, T = A.T, n = W * H * T;
    e = cudaMemsetAsync(A.acc, 0, QACC_WORDS * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (A.d2_a && (e = cudaMemsetAsync(A.d2_a, 0xff, n * sizeof(int32_t), st)) != cudaSuccess) return e;
    if (A.d2_b && (e = cudaMemsetAsync(A.d2_b, 0xff, n * sizeof(int32_t), st)) != cudaSuccess) return e;
    const int vec = ((reinterpret_cast<uintptr_t>(A.a) | reinterpret_cast<uintptr_t>(A.b)) & 15) == 0;
    k_frame_error<<<grid_of(n / 16 + 1, QBLOCK, sms, 8), QBLOCK, 0, st>>>(A.a, A.b, n, vec, A.acc);
    ++nl;
    // rows: warps per block bounded by the shared budget (W ints per warp)
    const int wpb = (int)std::max<int64_t>(1, std::min<int64_t>(8, SMEM_BUDGET / (4 * W)));
    auto cols_threads = [](int64_t L) {
        int64_t nt = SMEM_BUDGET / (8 * L);
        nt = nt >= 64 ? (nt / 32) * 32 : nt;
        return (int)std::max<int64_t>(1, std::min<int64_t>(256, nt));
    };
    for (int dir = 0; dir < 2; ++dir) {
        const int8_t* target = dir ? A.a : A.b;
        const int8_t* query = dir ? A.b : A.a;
        int32_t* d2_out = dir ? A.d2_b : A.d2_a;
        const int slot = dir ? QACC_MATCH_B : QACC_MATCH_A;
        for (int pol = 1; pol >= -1; pol -= 2) {
            int32_t* cur = A.vol0;
            int32_t* other = A.vol1;
            k_edt_rows<<<grid_of(H * T, wpb, sms, 16), 32 * wpb, (size_t)wpb * W * 4, st>>>(target, (int)W, H * T,
                                                                                            pol, cur);
            ++nl;
            // column passes along y, then t
            const int64_t lines[2] = {T * W, H * W}, ostride[2] = {H * W, W}, stp[2] = {W, H * W};
            const int64_t len[2] = {H, T};
            for (int ax = 0; ax < 2; ++ax) {
                if (len[ax] < 2) continue;
                const int L = (int)len[ax];
                const int blocks = stack_blocks(lines[ax], L, sms);
                k_edt_cols<<<blocks, 256, 0, st>>>(cur, other, lines[ax], (int)W, ostride[ax], stp[ax], L,
                                                    reinterpret_cast<int2*>(A.stack));
                ++nl;
                std::swap(cur, other);
            }
            const int qvec = (reinterpret_cast<uintptr_t>(query) & 3) == 0;
            k_match<<<grid_of(n / 4 + 1, QBLOCK, sms, 8), QBLOCK, 0, st>>>(
                query, cur, n, pol, A.tau2, qvec, d2_out, A.acc, slot, A.acc + (dir ? QACC_HIST_B : QACC_HIST_A));
            ++nl;
        }
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace mcev
