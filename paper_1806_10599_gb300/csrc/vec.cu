// Conjugate-gradient vector updates and reductions (Sect. 2.1, the Krylov
// solver of Eq. linequil2).  Reductions are two-stage and deterministic: a
// fixed grid of RED_BLOCKS blocks writes partial sums, one block adds them in
// a fixed order.  Sums are accumulated in FP64 for both precisions (FP32 data:
// each 4-element vector's part in FP32 first, see vdot_acc).
#include "gff_internal.cuh"

namespace gff {
namespace {

constexpr int TPB = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}

// 16-byte vectors of the CG kernels: every vector length here is a multiple of
// 4 (9 N with nx, ny even) and every base 16-byte aligned (cudaMalloc'd), so the
// streams are read and written as float4 / double2.  A thread takes whole
// vectors in a grid-stride loop and adds each vector's contribution to its FP64
// sum in order; the single-RVE and the batched kernels share this mapping, so
// their reductions are bitwise equal.
template <typename T> struct Vec;
template <> struct Vec<float> {
    using t = float4;
    static constexpr int n = 4;
};
template <> struct Vec<double> {
    using t = double2;
    static constexpr int n = 2;
};
template <typename T> __device__ __forceinline__ T& at(typename Vec<T>::t& v, int j) {
    return reinterpret_cast<T*>(&v)[j];
}
template <typename T> __device__ __forceinline__ T get(const typename Vec<T>::t& v, int j) {
    return reinterpret_cast<const T*>(&v)[j];
}

// a . b of one vector, added to the FP64 sum: FP64 products for double data; for
// float data the vector's products are summed in FP32 first (one conversion and
// one FP64 add per four elements -- conversions and FP64 FMAs per element would
// make the FP32 kernels FP64-pipe bound)
__device__ __forceinline__ double vdot_acc(const double2& x, const double2& y, double acc) {
    return fma(x.y, y.y, fma(x.x, y.x, acc));
}
__device__ __forceinline__ double vdot_acc(const float4& x, const float4& y, double acc) {
    return acc + (double)fmaf(x.w, y.w, fmaf(x.z, y.z, fmaf(x.y, y.y, x.x * y.x)));
}

template <typename T>
__device__ __forceinline__ double dot_thread(const T* __restrict__ a, const T* __restrict__ b, long long n) {
    using V = typename Vec<T>::t;
    constexpr int W = Vec<T>::n;
    const V* a4 = reinterpret_cast<const V*>(a);
    const V* b4 = reinterpret_cast<const V*>(b);
    const long long nv = n / W, gs = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + gs < nv; i += 2 * gs) {  // two vectors in flight per thread
        const V x0 = a4[i], y0 = b4[i], x1 = a4[i + gs], y1 = b4[i + gs];
        acc = vdot_acc(x0, y0, acc);
        acc = vdot_acc(x1, y1, acc);
    }
    if (i < nv) acc = vdot_acc(a4[i], b4[i], acc);
    return acc;
}

// x += alpha p, r -= alpha Ap; returns this thread's part of r.r
template <typename T>
__device__ __forceinline__ double update_thread(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                const T* __restrict__ Ap, T alpha, long long n) {
    using V = typename Vec<T>::t;
    constexpr int W = Vec<T>::n;
    V* x4 = reinterpret_cast<V*>(x);
    V* r4 = reinterpret_cast<V*>(r);
    const V* p4 = reinterpret_cast<const V*>(p);
    const V* a4 = reinterpret_cast<const V*>(Ap);
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n / W; i += (long long)gridDim.x * blockDim.x) {
        V xv = x4[i], rv = r4[i];
        const V pv = p4[i], av = a4[i];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            at<T>(xv, j) = fma(alpha, get<T>(pv, j), get<T>(xv, j));
            at<T>(rv, j) = fma(-alpha, get<T>(av, j), get<T>(rv, j));
        }
        acc = vdot_acc(rv, rv, acc);
        x4[i] = xv;
        r4[i] = rv;
    }
    return acc;
}

// p = r + beta p
template <typename T>
__device__ __forceinline__ void xpby_thread(T* __restrict__ p, const T* __restrict__ r, T beta, long long n) {
    using V = typename Vec<T>::t;
    constexpr int W = Vec<T>::n;
    V* p4 = reinterpret_cast<V*>(p);
    const V* r4 = reinterpret_cast<const V*>(r);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n / W; i += (long long)gridDim.x * blockDim.x) {
        V pv = p4[i];
        const V rv = r4[i];
#pragma unroll
        for (int j = 0; j < W; ++j) at<T>(pv, j) = fma(beta, get<T>(pv, j), get<T>(rv, j));
        p4[i] = pv;
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_dot_partial(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                                     double* __restrict__ partial) {
    __shared__ double sh[32];
    double acc = dot_thread<T>(a, b, n);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[k] = sum_b partial[k * nb + b], one block per k
__global__ void __launch_bounds__(TPB) k_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[(long long)blockIdx.x * nb + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// per-component sums of a [9][N] field: grid (RED_BLOCKS, 9)
__global__ void __launch_bounds__(TPB) k_sum9_partial(const double* __restrict__ a, long long N,
                                                      double* __restrict__ partial) {
    __shared__ double sh[32];
    const double2* ac = reinterpret_cast<const double2*>(a + (long long)blockIdx.y * N);  // N is a multiple of 4
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N / 2; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = ac[i];
        acc += v.x;
        acc += v.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_cg_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                   const T* __restrict__ Ap, T alpha, long long n,
                                                   double* __restrict__ partial) {
    __shared__ double sh[32];
    double acc = update_thread<T>(x, r, p, Ap, alpha, n);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_xpby(T* __restrict__ p, const T* __restrict__ r, T beta, long long n) {
    xpby_thread<T>(p, r, beta, n);
}

struct Nine {
    double v[9];
};

__global__ void __launch_bounds__(TPB) k_add_const9(double* __restrict__ F, const double* __restrict__ Fsrc, Nine d,
                                                    long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 9 * N; i += (long long)gridDim.x * blockDim.x)
        F[i] = Fsrc[i] + d.v[i / N];
}

__global__ void __launch_bounds__(TPB) k_fluct_incr(float* __restrict__ y, const double* __restrict__ Fk,
                                                    const double* __restrict__ F, Nine d, double inv, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 9 * N; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)((Fk[i] - F[i] - d.v[i / N]) * inv);
}

template <typename Tin>
__global__ void __launch_bounds__(TPB) k_axpy_to64(double* __restrict__ y, const Tin* __restrict__ x, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += (double)x[i];
}

__global__ void __launch_bounds__(TPB) k_cast(float* __restrict__ y, const double* __restrict__ x, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_fill(T* __restrict__ y, T v, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = v;
}

// ---- device-resident CG iteration (no host round trip per iteration)
// Each reduction's partial sums and its final sum share one launch: the block
// that takes the grid's last ticket (flag[CG_TICKET_*], returned to 0 by that
// block) adds the RED_BLOCKS partials in the same fixed order as the batched
// final kernels, so the scalars stay deterministic and bitwise equal to the
// batched solver's.  Three launches per iteration: p.Ap with alpha; the x, r
// update with r.r, beta and the convergence test; the direction update.
// The two reductions are bounded to RED_BLOCKS / 152 resident blocks per SM
// (64 registers): with fewer, a second wave of blocks would run their
// grid-stride loops alone.
__global__ void k_cg_init(double* cg, int* flag, double rr0, double stop2) {
    cg[CG_RR] = rr0;
    cg[CG_PAP] = 0.0;
    cg[CG_ALPHA] = 0.0;
    cg[CG_BETA] = 0.0;
    cg[CG_STOP2] = stop2;
    cg[CG_ITERS] = 0.0;
    flag[0] = rr0 <= stop2 ? 1 : 0;
    flag[1] = 0;
    flag[CG_TICKET_ALPHA] = flag[CG_TICKET_BETA] = 0;
}

// True in every thread of the block that finishes last; every other block's
// partial sum (stored before its ticket, behind a fence) is then visible.
__device__ __forceinline__ bool last_block(int* ticket) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
        if (last) *ticket = 0;
    }
    __syncthreads();
    return last != 0;
}

// the sum of nb partials, in the order of the batched final kernels (L2 reads:
// the partials were written by other blocks of this launch)
__device__ __forceinline__ double partial_total(const double* partial, int nb, double* sh) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += __ldcg(partial + i);
    return block_sum(acc, sh);
}

// p.Ap, then (last block) alpha = r.r / p.Ap; a zero or non-finite p.Ap stops
// the solve with the breakdown flag
template <typename T>
__global__ void __launch_bounds__(TPB, RED_BLOCKS / 152) k_cg_alpha(const T* __restrict__ p, const T* __restrict__ Ap, long long n,
                                                 double* __restrict__ partial, double* cg, int* flag) {
    if (*flag) {
        // a stop reached in the previous iteration (2: its direction update has run) becomes final
        if (blockIdx.x == 0 && threadIdx.x == 0 && *flag == 2) *flag = 1;
        return;
    }
    __shared__ double sh[32];
    double acc = block_sum(dot_thread<T>(p, Ap, n), sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    if (!last_block(flag + CG_TICKET_ALPHA)) return;
    acc = partial_total(partial, gridDim.x, sh);
    if (threadIdx.x == 0) {
        cg[CG_PAP] = acc;
        if (acc == 0.0 || !isfinite(acc)) {
            flag[1] = 1;
            flag[0] = 1;
        } else {
            cg[CG_ALPHA] = cg[CG_RR] / acc;
        }
    }
}

// x += alpha p, r -= alpha Ap with r.r, then (last block) beta = r.r(new) /
// r.r(old), the iteration count and the convergence test r.r <= stop^2
template <typename T>
__global__ void __launch_bounds__(TPB, RED_BLOCKS / 152) k_cg_update_dev(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                       const T* __restrict__ Ap, long long n, double* __restrict__ partial,
                                                       double* cg, int* flag) {
    if (*flag) return;
    __shared__ double sh[32];
    double acc = update_thread<T>(x, r, p, Ap, (T)cg[CG_ALPHA], n);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    if (!last_block(flag + CG_TICKET_BETA)) return;
    acc = partial_total(partial, gridDim.x, sh);
    if (threadIdx.x == 0) {
        cg[CG_BETA] = acc / cg[CG_RR];
        cg[CG_RR] = acc;
        cg[CG_ITERS] += 1.0;
        if (!isfinite(acc)) {
            flag[1] = 1;
            flag[0] = 1;
        } else if (acc <= cg[CG_STOP2]) {
            flag[0] = 2;  // converged; the direction update below still runs this once
        }
    }
}

// p = r + beta p (skipped once the solve has stopped before this iteration;
// flag 2, convergence in this iteration, still runs it -- the next k_cg_alpha
// makes the stop final)
template <typename T>
__global__ void __launch_bounds__(TPB) k_xpby_dev(T* __restrict__ p, const T* __restrict__ r, long long n,
                                                  const double* __restrict__ cg, const int* __restrict__ flag) {
    if (*flag == 1) return;
    xpby_thread<T>(p, r, (T)cg[CG_BETA], n);
}

// ---- batched CG: blockIdx.y = RVE; each RVE uses the same RED_BLOCKS x TPB
// grid-stride pattern as the single-RVE kernels, so its sums are bitwise equal
template <typename T>
__global__ void __launch_bounds__(TPB) k_dot_partial_batch(const RveVec* __restrict__ v, int which,
                                                           double* __restrict__ partial, const int* __restrict__ flag) {
    const int r = blockIdx.y;
    if (flag && flag[2 * r]) return;
    __shared__ double sh[32];
    const T* a = static_cast<const T*>(which == 0 ? v[r].p : v[r].x);
    const T* b = static_cast<const T*>(which == 0 ? v[r].Ap : v[r].r);
    double acc = dot_thread<T>(a, b, v[r].n);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(TPB) k_final_alpha_batch(const double* __restrict__ partial, int nb, double* cg,
                                                           int* flag) {
    const int r = blockIdx.x;
    if (flag[2 * r]) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[(long long)r * nb + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double* c = cg + 8 * r;
        c[CG_PAP] = acc;
        if (acc == 0.0 || !isfinite(acc)) {
            flag[2 * r + 1] = 1;
            flag[2 * r] = 1;
        } else {
            c[CG_ALPHA] = c[CG_RR] / acc;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_cg_update_batch(const RveVec* __restrict__ v, double* __restrict__ partial,
                                                         const double* __restrict__ cg, const int* __restrict__ flag) {
    const int r = blockIdx.y;
    if (flag[2 * r]) return;
    __shared__ double sh[32];
    double acc = update_thread<T>(static_cast<T*>(v[r].x), static_cast<T*>(v[r].r), static_cast<const T*>(v[r].p),
                                  static_cast<const T*>(v[r].Ap), (T)cg[8 * r + CG_ALPHA], v[r].n);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(TPB) k_final_beta_batch(const double* __restrict__ partial, int nb, double* cg,
                                                          int* flag) {
    const int r = blockIdx.x;
    if (flag[2 * r]) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[(long long)r * nb + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double* c = cg + 8 * r;
        c[CG_BETA] = acc / c[CG_RR];
        c[CG_RR] = acc;
        c[CG_ITERS] += 1.0;
        if (!isfinite(acc)) {
            flag[2 * r + 1] = 1;
            flag[2 * r] = 1;
        } else if (acc <= c[CG_STOP2]) {
            flag[2 * r] = 2;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_xpby_batch(const RveVec* __restrict__ v, const double* __restrict__ cg,
                                                    const int* __restrict__ flag) {
    const int r = blockIdx.y;
    if (flag[2 * r] == 1) return;
    xpby_thread<T>(static_cast<T*>(v[r].p), static_cast<const T*>(v[r].r), (T)cg[8 * r + CG_BETA], v[r].n);
}

__global__ void k_promote_stop_batch(int* flag, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n && flag[2 * r] == 2) flag[2 * r] = 1;
}

// rr0_stop2[2 r] = r.r of RVE r, [2 r + 1] = stop^2; rr0 < 0 marks an RVE that does not solve
__global__ void k_cg_init_batch(int n, double* cg, int* flag, const double* rr0_stop2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double rr0 = rr0_stop2[2 * r], s2 = rr0_stop2[2 * r + 1];
    double* c = cg + 8 * r;
    c[CG_RR] = rr0;
    c[CG_PAP] = 0.0;
    c[CG_ALPHA] = 0.0;
    c[CG_BETA] = 0.0;
    c[CG_STOP2] = s2;
    c[CG_ITERS] = 0.0;
    flag[2 * r] = (rr0 < 0.0 || rr0 <= s2) ? 1 : 0;
    flag[2 * r + 1] = 0;
}

inline int grid_for(long long n) {
    long long b = (n + TPB - 1) / TPB;
    return (int)(b < 152LL * 8 ? (b < 1 ? 1 : b) : 152LL * 8);
}

}  // namespace

template <typename T>
cudaError_t launch_dot(const T* a, const T* b, long long n, double* partial, double* out, cudaStream_t s) {
    k_dot_partial<T><<<RED_BLOCKS, TPB, 0, s>>>(a, b, n, partial);
    k_final<<<1, TPB, 0, s>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}

cudaError_t launch_sum9(const double* a, long long N, double* partial, double* out9, cudaStream_t s) {
    k_sum9_partial<<<dim3(RED_BLOCKS, 9), TPB, 0, s>>>(a, N, partial);
    k_final<<<9, TPB, 0, s>>>(partial, RED_BLOCKS, out9);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(T* x, T* r, const T* p, const T* Ap, double alpha, long long n, double* partial,
                             double* out_rr, cudaStream_t s) {
    k_cg_update<T><<<RED_BLOCKS, TPB, 0, s>>>(x, r, p, Ap, (T)alpha, n, partial);
    k_final<<<1, TPB, 0, s>>>(partial, RED_BLOCKS, out_rr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xpby(T* p, const T* r, double beta, long long n, cudaStream_t s) {
    k_xpby<T><<<grid_for(n), TPB, 0, s>>>(p, r, (T)beta, n);
    return cudaGetLastError();
}

cudaError_t launch_add_const9(double* F, const double* Fsrc, const double* d9, long long N, cudaStream_t s) {
    Nine d;
    for (int c = 0; c < 9; ++c) d.v[c] = d9[c];
    k_add_const9<<<grid_for(9 * N), TPB, 0, s>>>(F, Fsrc, d, N);
    return cudaGetLastError();
}

template <typename Tin>
cudaError_t launch_axpy_to64(double* y, const Tin* x, long long n, cudaStream_t s) {
    k_axpy_to64<Tin><<<grid_for(n), TPB, 0, s>>>(y, x, n);
    return cudaGetLastError();
}

cudaError_t launch_fluct_incr(float* y, const double* Fk, const double* F, const double* dF9, double inv, long long N,
                              cudaStream_t s) {
    Nine d;
    for (int c = 0; c < 9; ++c) d.v[c] = dF9[c];
    k_fluct_incr<<<grid_for(9 * N), TPB, 0, s>>>(y, Fk, F, d, inv, N);
    return cudaGetLastError();
}

cudaError_t launch_cast64to32(float* y, const double* x, long long n, cudaStream_t s) {
    k_cast<<<grid_for(n), TPB, 0, s>>>(y, x, n);
    return cudaGetLastError();
}

cudaError_t launch_fill(double* y, double v, long long n, cudaStream_t s) {
    k_fill<double><<<grid_for(n), TPB, 0, s>>>(y, v, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(T* y, long long n, cudaStream_t s) {
    k_fill<T><<<grid_for(n), TPB, 0, s>>>(y, (T)0, n);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(double* cg, int* flag, double rr0, double stop2, cudaStream_t s) {
    k_cg_init<<<1, 1, 0, s>>>(cg, flag, rr0, stop2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_alpha(const T* p, const T* Ap, long long n, double* partial, double* cg, int* flag,
                            cudaStream_t s) {
    k_cg_alpha<T><<<RED_BLOCKS, TPB, 0, s>>>(p, Ap, n, partial, cg, flag);
    return cudaGetLastError();
}

// x += alpha p, r -= alpha Ap, r.r, beta, convergence test, p = r + beta p
template <typename T>
cudaError_t launch_cg_step(T* x, T* r, T* p, const T* Ap, long long n, double* partial, double* cg, int* flag,
                           cudaStream_t s) {
    k_cg_update_dev<T><<<RED_BLOCKS, TPB, 0, s>>>(x, r, p, Ap, n, partial, cg, flag);
    k_xpby_dev<T><<<grid_for(n), TPB, 0, s>>>(p, r, n, cg, flag);
    return cudaGetLastError();
}

// ---- measurement helpers

namespace {
// Independent FP64 FMA chains: 8 per thread, `iters` rounds each.  The
// constants keep every chain bounded (x -> b / (1 - a)); the final store keeps
// the work alive.
__global__ void __launch_bounds__(256) k_fma64_chains(double* __restrict__ out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-6, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
    double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_fill_ramp(T* __restrict__ y, long long n, double base) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)(base + 1e-3 * (double)(i & 1023));
}
}  // namespace

// FP64 FMA throughput of this GPU: blocks x 256 threads x 8 chains x iters
// FMAs (2 flops each), timed with CUDA events on stream s.  out holds blocks x
// 256 doubles.  The best of `reps` launches is returned.
cudaError_t measure_fp64_fma(double* out, int blocks, int iters, int reps, cudaStream_t s, double* gflops,
                             float* ms_best) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    k_fma64_chains<<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-6);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) k_fma64_chains<<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-6);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    *ms_best = best;
    *gflops = 2.0 * 8.0 * (double)blocks * 256.0 * (double)iters / (best * 1e-3) / 1e9;
    return cudaSuccess;
}

// Times the CG vector kernels of one iteration on the vectors x, r, p, Ap
// (n elements, overwritten with a ramp first): ms[0] p.Ap (partial sums and
// alpha), ms[1] x += alpha p, r -= alpha Ap with r.r (and beta), ms[2]
// p = r + beta p; averages over `reps` iterations.
template <typename T>
cudaError_t time_cg_kernels(T* x, T* r, T* p, T* Ap, long long n, double* partial, double* cg, int* flag,
                            cudaStream_t s, int reps, float* ms) {
    const int gb = grid_for(n);
    k_fill_ramp<T><<<gb, TPB, 0, s>>>(x, n, 0.0);
    k_fill_ramp<T><<<gb, TPB, 0, s>>>(r, n, 1.0);
    k_fill_ramp<T><<<gb, TPB, 0, s>>>(p, n, 1.0);
    k_fill_ramp<T><<<gb, TPB, 0, s>>>(Ap, n, 2.0);
    k_cg_init<<<1, 1, 0, s>>>(cg, flag, 1.0, 0.0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; ++i)
        if ((e = cudaEventCreate(&ev[i])) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return e;
        }
    double acc[3] = {0, 0, 0};
    for (int it = 0; it < reps && e == cudaSuccess; ++it) {
        cudaEventRecord(ev[0], s);
        k_cg_alpha<T><<<RED_BLOCKS, TPB, 0, s>>>(p, Ap, n, partial, cg, flag);
        cudaEventRecord(ev[1], s);
        k_cg_update_dev<T><<<RED_BLOCKS, TPB, 0, s>>>(x, r, p, Ap, n, partial, cg, flag);
        cudaEventRecord(ev[2], s);
        k_xpby_dev<T><<<grid_for(n), TPB, 0, s>>>(p, r, n, cg, flag);
        cudaEventRecord(ev[3], s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / (reps > 0 ? reps : 1));
    return e;
}
template cudaError_t time_cg_kernels<double>(double*, double*, double*, double*, long long, double*, double*, int*,
                                             cudaStream_t, int, float*);
template cudaError_t time_cg_kernels<float>(float*, float*, float*, float*, long long, double*, double*, int*,
                                            cudaStream_t, int, float*);

template cudaError_t launch_cg_alpha<double>(const double*, const double*, long long, double*, double*, int*,
                                             cudaStream_t);
template cudaError_t launch_cg_alpha<float>(const float*, const float*, long long, double*, double*, int*,
                                            cudaStream_t);
template cudaError_t launch_cg_step<double>(double*, double*, double*, const double*, long long, double*, double*,
                                            int*, cudaStream_t);
template cudaError_t launch_cg_step<float>(float*, float*, float*, const float*, long long, double*, double*, int*,
                                           cudaStream_t);

cudaError_t launch_cg_init_batch(int n, double* cg, int* flag, const double* rr0_stop2_dev, cudaStream_t s) {
    k_cg_init_batch<<<(n + 63) / 64, 64, 0, s>>>(n, cg, flag, rr0_stop2_dev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_alpha_batch(int n, const RveVec* v, double* partial, double* cg, int* flag, cudaStream_t s) {
    k_dot_partial_batch<T><<<dim3(RED_BLOCKS, n), TPB, 0, s>>>(v, 0, partial, flag);
    k_final_alpha_batch<<<n, TPB, 0, s>>>(partial, RED_BLOCKS, cg, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_step_batch(int n, const RveVec* v, double* partial, double* cg, int* flag, cudaStream_t s) {
    k_cg_update_batch<T><<<dim3(RED_BLOCKS, n), TPB, 0, s>>>(v, partial, cg, flag);
    k_final_beta_batch<<<n, TPB, 0, s>>>(partial, RED_BLOCKS, cg, flag);
    k_xpby_batch<T><<<dim3(RED_BLOCKS, n), TPB, 0, s>>>(v, cg, flag);
    k_promote_stop_batch<<<(n + 63) / 64, 64, 0, s>>>(flag, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dot_batch(int n, const RveVec* v, double* partial, double* out, cudaStream_t s) {
    k_dot_partial_batch<T><<<dim3(RED_BLOCKS, n), TPB, 0, s>>>(v, 1, partial, nullptr);
    k_final<<<n, TPB, 0, s>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}

template cudaError_t launch_cg_alpha_batch<double>(int, const RveVec*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_cg_alpha_batch<float>(int, const RveVec*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_cg_step_batch<double>(int, const RveVec*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_cg_step_batch<float>(int, const RveVec*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_dot_batch<double>(int, const RveVec*, double*, double*, cudaStream_t);
template cudaError_t launch_dot_batch<float>(int, const RveVec*, double*, double*, cudaStream_t);

template cudaError_t launch_dot<double>(const double*, const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_dot<float>(const float*, const float*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_cg_update<double>(double*, double*, const double*, const double*, double, long long,
                                              double*, double*, cudaStream_t);
template cudaError_t launch_cg_update<float>(float*, float*, const float*, const float*, double, long long, double*,
                                             double*, cudaStream_t);
template cudaError_t launch_xpby<double>(double*, const double*, double, long long, cudaStream_t);
template cudaError_t launch_xpby<float>(float*, const float*, double, long long, cudaStream_t);
template cudaError_t launch_axpy_to64<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t launch_axpy_to64<float>(double*, const float*, long long, cudaStream_t);
template cudaError_t launch_zero<double>(double*, long long, cudaStream_t);
template cudaError_t launch_zero<float>(float*, long long, cudaStream_t);

}  // namespace gff
