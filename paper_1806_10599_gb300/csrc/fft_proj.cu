// Galerkin operator y = F^-1{ G^ : F(K : x) }  (Eqs. eql_discrete3, newlinop)
// as three kernels over the [9][nz][ny][nx] field:
//
//   k_plane_fwd  one CTA per (component c, plane z): optional per-voxel
//                contraction y_c = K_cd x_d, then the 2D forward transform of
//                the plane held in shared memory -- a real-to-complex pass
//                along x (two real rows packed as one complex row) and a
//                complex pass along y -- written as the half spectrum
//                [9][nz][ny][nx/2+1].
//   k_zproj      one CTA per W consecutive (ky, kx) columns: forward
//                transform along z of all 9 components, the projection
//                G^ (Eq. G) or G^' (Sect. 2.2) at every frequency, inverse
//                transform along z, in place.
//   k_plane_inv  one CTA per (c, z): inverse y, complex-to-real x, epilogue
//                out = scale * y + add_c.
//
// Each axis transform is an in-place mixed-radix (2, 3, 4, 5, 8, 16) FFT in
// shared memory: forward = decimation in frequency (natural order in,
// digit-reversed out), inverse = the same stages replayed backwards with
// conjugate twiddles (digit-reversed in, natural out), so no reordering pass
// is needed; the projection reads the frequency of each position from a table.
// The common lengths (16 ... 128) have two-stage plans with compile-time
// radices (fft2_lines); the others run the generic stages.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "bulk_copy.cuh"
#include "gff_internal.cuh"

namespace gff {
namespace {

template <typename C>
__device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// a * w and a * conj(w)
template <typename C> __device__ __forceinline__ C cmul(C a, C w) {
    return mk<C>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C w) {
    return mk<C>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
    return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// ---------------------------------------------------------------- butterflies
// Unnormalised radix-R DFT of v[0..R-1]: y_p = sum_q v_q w^(pq), w = exp(-+2 pi i / R).
template <int R, bool INV, typename C> struct Bfly;

template <bool INV, typename C> struct Bfly<2, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV, typename C> struct Bfly<4, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        C a2 = cadd(v[1], v[3]), a3 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
};

template <bool INV, typename C> struct Bfly<8, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        using T = decltype(C::x);
        const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Bfly<4, INV, C>::run(e);
        Bfly<4, INV, C>::run(o);
        // o_p *= w8^p, w8 = exp(-+ i pi / 4)
        C o1 = INV ? mk<C>((o[1].x - o[1].y) * h, (o[1].x + o[1].y) * h)
                   : mk<C>((o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h);
        C o2 = rot90<INV>(o[2]);
        C o3 = INV ? mk<C>(-(o[3].x + o[3].y) * h, (o[3].x - o[3].y) * h)
                   : mk<C>((o[3].y - o[3].x) * h, -(o[3].x + o[3].y) * h);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <bool INV, typename C> struct Bfly<3, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        using T = decltype(C::x);
        const T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = csub(v[0], cscale(t1, (T)0.5));
        C t3 = rot90<INV>(cscale(csub(v[1], v[2]), s3));  // -+ i s3 (v1 - v2)
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};

template <bool INV, typename C> struct Bfly<5, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        using T = decltype(C::x);
        const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
        const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
        const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
        const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
        C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        C a1 = mk<C>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        C a2 = mk<C>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        C b1 = rot90<INV>(mk<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        C b2 = rot90<INV>(mk<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

// a * (c -+ i s): multiplication by a constant twiddle exp(-+ i theta), c = cos, s = sin
template <bool INV, typename C, typename T>
__device__ __forceinline__ C twc(C a, T c, T s) {
    return INV ? mk<C>(a.x * c - a.y * s, a.y * c + a.x * s) : mk<C>(a.x * c + a.y * s, a.y * c - a.x * s);
}

// radix 16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2,
// X[k1 + 4 k2] = sum_n2 w4^(n2 k2) w16^(n2 k1) sum_n1 x[4 n1 + n2] w4^(n1 k1)
template <bool INV, typename C> struct Bfly<16, INV, C> {
    static __device__ __forceinline__ void run(C* v) {
        using T = decltype(C::x);
        const T c1 = (T)0.92387953251128675613;  // cos(pi / 8)
        const T s1 = (T)0.38268343236508977173;  // sin(pi / 8)
        const T h = (T)0.70710678118654752440;   // cos(pi / 4)
        C y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            C a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
            Bfly<4, INV, C>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
        }
        // w16^m for m = n2 k1: 1 (c1, s1), 2 (h, h), 3 (s1, c1), 4 (-+ i), 6 (-h, h), 9 (-c1, -s1)
        y[1][1] = twc<INV>(y[1][1], c1, s1);
        y[1][2] = twc<INV>(y[1][2], h, h);
        y[1][3] = twc<INV>(y[1][3], s1, c1);
        y[2][1] = twc<INV>(y[2][1], h, h);
        y[2][2] = rot90<INV>(y[2][2]);
        y[2][3] = twc<INV>(y[2][3], -h, h);
        y[3][1] = twc<INV>(y[3][1], s1, c1);
        y[3][2] = twc<INV>(y[3][2], -h, h);
        y[3][3] = twc<INV>(y[3][3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C b[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Bfly<4, INV, C>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
        }
    }
};

// ---------------------------------------------------------------- one radix stage
// Lines l = ls * NLF + lf start at s + ls*SS + lf*SF; elements are ES apart.
// Sub-arrays of length `len` are split by radix R with stride m = len / R.
// Threads take (lf fastest, then butterfly, then ls) so that neighbouring
// lanes touch neighbouring shared-memory words.
template <typename T, int R, bool INV>
__device__ __forceinline__ void run_stage(typename C2<T>::t* s, const typename C2<T>::t* tw, int n, int len,
                                          int NLF, int SF, int NLS, int SS, int ES, int tid, int nthr) {
    using C = typename C2<T>::t;
    const int m = len / R, nb = n / R, twstep = n / len;
    const int total = NLF * nb * NLS;
    const int st = m * ES;
    for (int idx = tid; idx < total; idx += nthr) {
        const int lf = idx % NLF;
        const int t = idx / NLF;
        const int bb = t % nb;
        const int lsl = t / nb;
        const int sub = bb / m;
        const int j = bb - sub * m;
        C* base = s + lsl * SS + lf * SF + (sub * len + j) * ES;
        C v[R];
        if (!INV) {
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = base[q * st];
            Bfly<R, false, C>::run(v);
            if (j) {
#pragma unroll
                for (int p = 1; p < R; ++p) v[p] = cmul(v[p], tw[p * j * twstep]);
            }
#pragma unroll
            for (int p = 0; p < R; ++p) base[p * st] = v[p];
        } else {
#pragma unroll
            for (int p = 0; p < R; ++p) v[p] = base[p * st];
            if (j) {
#pragma unroll
                for (int p = 1; p < R; ++p) v[p] = cmulc(v[p], tw[p * j * twstep]);
            }
            Bfly<R, true, C>::run(v);
#pragma unroll
            for (int q = 0; q < R; ++q) base[q * st] = v[q];
        }
    }
}

template <typename T, bool INV>
__device__ __forceinline__ void stage_dispatch(int R, typename C2<T>::t* s, const typename C2<T>::t* tw, int n,
                                               int len, int NLF, int SF, int NLS, int SS, int ES, int tid,
                                               int nthr) {
    switch (R) {
        case 16: run_stage<T, 16, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        case 8: run_stage<T, 8, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        case 4: run_stage<T, 4, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        case 2: run_stage<T, 2, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        case 3: run_stage<T, 3, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        case 5: run_stage<T, 5, INV>(s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr); break;
        default: break;
    }
}

// q = x / d, r = x - q d for 0 <= x < 2^22 and d >= 1 (invd = 1 / d as float):
// the float quotient is within one of the true one, and one correction fixes it.
__device__ __forceinline__ int divmod_f(int x, int d, float invd, int& r) {
    int q = __float2int_rz(__int2float_rn(x) * invd);
    r = x - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}

// Two-stage transform of length N = R1 R2 (the plans of the common sizes):
// the radix-R1 stage over stride R2 with twiddles w_N^(p j), then radix R2
// over contiguous runs without twiddles -- the generic stages below with
// compile-time radices and one (float) division per butterfly.
template <typename T, int R1, int R2, bool TWIDDLED, bool INV>
__device__ __forceinline__ void fft2_stage(typename C2<T>::t* s, const typename C2<T>::t* tw, int NLF, float invNLF,
                                           int SF, int NLS, int SS, int ES, int tid, int nthr) {
    using C = typename C2<T>::t;
    // TWIDDLED: radix R1, tasks j < R2, elements j + q R2; else radix R2, tasks sub < R1, elements sub R2 + q
    constexpr int R = TWIDDLED ? R1 : R2;
    constexpr int TASKS = TWIDDLED ? R2 : R1;
    const int total = NLF * TASKS * NLS;
    const int st = (TWIDDLED ? R2 : 1) * ES;
    for (int idx = tid; idx < total; idx += nthr) {
        int lf = 0, t = idx;
        if (NLF > 1) t = divmod_f(idx, NLF, invNLF, lf);
        const int task = t % TASKS, lsl = t / TASKS;
        C* base = s + lsl * SS + lf * SF + (TWIDDLED ? task : task * R2) * ES;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = base[q * st];
        if (TWIDDLED && INV && task) {
#pragma unroll
            for (int p = 1; p < R; ++p) v[p] = cmulc(v[p], tw[p * task]);
        }
        Bfly<R, INV, C>::run(v);
        if (TWIDDLED && !INV && task) {
#pragma unroll
            for (int p = 1; p < R; ++p) v[p] = cmul(v[p], tw[p * task]);
        }
#pragma unroll
        for (int p = 0; p < R; ++p) base[p * st] = v[p];
    }
}

template <typename T, int R1, int R2, bool INV>
__device__ __forceinline__ void fft2_lines(typename C2<T>::t* s, const typename C2<T>::t* tw, int NLF, int SF,
                                           int NLS, int SS, int ES, int tid, int nthr) {
    const float invNLF = 1.0f / (float)NLF;
    if (!INV) {
        fft2_stage<T, R1, R2, true, false>(s, tw, NLF, invNLF, SF, NLS, SS, ES, tid, nthr);
        __syncthreads();
        fft2_stage<T, R1, R2, false, false>(s, tw, NLF, invNLF, SF, NLS, SS, ES, tid, nthr);
    } else {
        fft2_stage<T, R1, R2, false, true>(s, tw, NLF, invNLF, SF, NLS, SS, ES, tid, nthr);
        __syncthreads();
        fft2_stage<T, R1, R2, true, true>(s, tw, NLF, invNLF, SF, NLS, SS, ES, tid, nthr);
    }
    __syncthreads();
}

// Whole transform of a batch of lines; ends with a barrier.  Not inlined:
// every kernel calls the same four instances (precision x direction).
template <typename T, bool INV>
__device__ __noinline__ void fft_lines(typename C2<T>::t* s, const typename C2<T>::t* tw, const AxisPlan& pl, int NLF, int SF,
                          int NLS, int SS, int ES, int tid, int nthr) {
    const int n = pl.n;
    if (pl.nst == 2) {
        const int r1 = pl.radix[0], r2 = pl.radix[1];
#define GFF_FFT2(A, B)                                                                  \
    if (r1 == A && r2 == B) {                                                           \
        fft2_lines<T, A, B, INV>(s, tw, NLF, SF, NLS, SS, ES, tid, nthr);               \
        return;                                                                         \
    }
        GFF_FFT2(16, 8)
        GFF_FFT2(8, 8)
        GFF_FFT2(16, 5)
        GFF_FFT2(16, 3)
        GFF_FFT2(8, 5)
        GFF_FFT2(8, 4)
        GFF_FFT2(8, 3)
        GFF_FFT2(4, 4)
#undef GFF_FFT2
    }
    if (!INV) {
        int len = n;
        for (int k = 0; k < pl.nst; ++k) {
            stage_dispatch<T, false>(pl.radix[k], s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr);
            len /= pl.radix[k];
            __syncthreads();
        }
    } else {
        int len = 1;
        for (int k = pl.nst - 1; k >= 0; --k) {
            len *= pl.radix[k];
            stage_dispatch<T, true>(pl.radix[k], s, tw, n, len, NLF, SF, NLS, SS, ES, tid, nthr);
            __syncthreads();
        }
    }
}

template <typename T> __device__ __forceinline__ const typename C2<T>::t* twp(const GridDev& g, int a);
template <> __device__ __forceinline__ const double2* twp<double>(const GridDev& g, int a) { return g.tw64[a]; }
template <> __device__ __forceinline__ const float2* twp<float>(const GridDev& g, int a) { return g.tw32[a]; }
template <typename T> __device__ __forceinline__ const T* qtp(const GridDev& g, int kind, int a);
template <> __device__ __forceinline__ const double* qtp<double>(const GridDev& g, int kind, int a) {
    return g.qt64[kind][a];
}
template <> __device__ __forceinline__ const float* qtp<float>(const GridDev& g, int kind, int a) {
    return g.qt32[kind][a];
}

// ---------------------------------------------------------------- pass 1: (K:x) and the 2D forward transform
// 16-byte vectors of T for the streaming loads and stores
template <typename T> struct V16;
template <> struct V16<double> {
    using t = double2;
    static constexpr int n = 2;
    static __device__ __forceinline__ double get(const double2& v, int j) { return j ? v.y : v.x; }
};
template <> struct V16<float> {
    using t = float4;
    static constexpr int n = 4;
    static __device__ __forceinline__ float get(const float4& v, int j) {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    }
};

// Split (pass 1) and merge (pass 3) of the packed rows: a warp takes SPLIT_ROWS
// packed rows, each lane one row and the frequencies k = kg + SPLIT_G t.  The
// positions of k after the x transform are digit-reversed (neighbouring k lie 8
// or 16 values apart), so lanes spread over rows as well as over k keep the
// shared-memory accesses at most 2-way conflicted in FP32.  FP64 keeps one row
// per warp: several rows per warp would not fit its register budget.
template <typename T> constexpr int SPLIT_ROWS = sizeof(T) == 4 ? 4 : 1;
template <typename T> constexpr int SPLIT_G = 32 / SPLIT_ROWS<T>;
template <typename T> constexpr int SPLIT_K = (MAXN / 2 + SPLIT_G<T>) / SPLIT_G<T>;  // covers k = 0 .. MAXN/2

// (K:x)_c (or x_c alone) of plane z written as ny/2 packed complex rows: row pair r
// (real part row 2r, imaginary part row 2r+1) at s + 2 r ls.
template <typename T, bool WITH_K, bool VEC>
__device__ __forceinline__ void plane_contract(typename C2<T>::t* s, const T* __restrict__ x, const T* __restrict__ K,
                                               const GridDev& g, const int c, const int z, const int ls) {
    using C = typename C2<T>::t;
    const int nx = g.nx, ny = g.ny, half = ny / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long N = g.N;
    const long long pl = (long long)z * ny * nx;
    if (VEC) {
        // 16-byte loads of VW consecutive voxels of one row; K row c is read
        // once, the 9 components of x are shared by the 9 CTAs of this plane.
        // Lanes 2i and 2i+1 take the same VW voxels of rows 2r and 2r+1 (the
        // real and imaginary parts of packed row r) and swap halves, so that
        // each writes VW/2 whole complex values -- one 16-byte shared-memory
        // store, contiguous across the warp.
        using VT = typename V16<T>::t;
        constexpr int VW = V16<T>::n, HW = VW / 2;
        const int nxv = nx / VW, total = ny * nxv;  // total is even
        const int lane = tid & 31;
        for (int e0 = tid - lane; e0 < total; e0 += nthr) {  // warp-uniform trip count
            const int e = e0 + lane;
            const bool act = e < total;  // the partner e ^ 1 is active too
            const int p = e & 1, q = e >> 1;
            const int r = q / nxv, xv = q - r * nxv;
            const long long v0 = pl + (long long)(2 * r + p) * nx + xv * VW;
            T acc[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) acc[j] = (T)0;
            if (act) {
                if (WITH_K) {
                    const T* Kc = K + (long long)c * 9 * N;
                    VT kv[9], xq[9];
#pragma unroll
                    for (int d = 0; d < 9; ++d) {
                        kv[d] = __ldg(reinterpret_cast<const VT*>(Kc + d * N + v0));
                        xq[d] = __ldg(reinterpret_cast<const VT*>(x + d * N + v0));
                    }
#pragma unroll
                    for (int j = 0; j < VW; ++j) {
                        T t = (T)0;
#pragma unroll
                        for (int d = 0; d < 9; ++d) t = fma(V16<T>::get(kv[d], j), V16<T>::get(xq[d], j), t);
                        acc[j] = t;
                    }
                } else {
                    const VT xv4 = __ldg(reinterpret_cast<const VT*>(x + c * N + v0));
#pragma unroll
                    for (int j = 0; j < VW; ++j) acc[j] = V16<T>::get(xv4, j);
                }
            }
            // lane p = 0 keeps voxels 0..HW-1 and receives their imaginary parts;
            // lane p = 1 keeps voxels HW..VW-1 and receives their real parts
            VT o;
            T* op = reinterpret_cast<T*>(&o);
#pragma unroll
            for (int j = 0; j < HW; ++j) {
                const T recv = __shfl_xor_sync(0xffffffffu, p ? acc[j] : acc[HW + j], 1);
                op[2 * j] = p ? recv : acc[j];
                op[2 * j + 1] = p ? acc[HW + j] : recv;
            }
            if (act) *reinterpret_cast<VT*>(s + r * 2 * ls + xv * VW + p * HW) = o;
        }
    } else {
        for (int e = tid; e < half * nx; e += nthr) {
            const int r = e / nx, xi = e - r * nx;
            const long long v0 = pl + (long long)(2 * r) * nx + xi, v1 = v0 + nx;
            T a, b;
            if (WITH_K) {
                a = (T)0;
                b = (T)0;
                const T* Kc = K + (long long)c * 9 * N;
#pragma unroll
                for (int d = 0; d < 9; ++d) {
                    a = fma(__ldg(Kc + d * N + v0), __ldg(x + d * N + v0), a);
                    b = fma(__ldg(Kc + d * N + v1), __ldg(x + d * N + v1), b);
                }
            } else {
                a = __ldg(x + c * N + v0);
                b = __ldg(x + c * N + v1);
            }
            s[r * 2 * ls + xi] = mk<C>(a, b);
        }
    }
}

template <typename T, bool WITH_K, bool VEC>
__device__ __forceinline__ void plane_fwd_body(const T* __restrict__ x, const T* __restrict__ K,
                                               typename C2<T>::t* __restrict__ spec, const GridDev& g, const int c,
                                               const int z, unsigned char* sm_raw) {
    using C = typename C2<T>::t;
    const int nx = g.nx, ny = g.ny, nxh = g.nxh, ls = nxh, half = ny / 2;
    C* s = reinterpret_cast<C*>(sm_raw);
    C* twx = s + ny * ls;
    C* twy = twx + nx;
    int* posx = reinterpret_cast<int*>(twy + ny);
    int* posy = posx + nx;  // position of each y frequency after the forward y transform
    const int tid = threadIdx.x, nthr = blockDim.x;

    for (int i = tid; i < nx; i += nthr) {
        twx[i] = twp<T>(g, 0)[i];
        posx[i] = g.posx[i];
    }
    for (int i = tid; i < ny; i += nthr) {
        twy[i] = twp<T>(g, 1)[i];
        posy[g.fqy[i]] = i;
    }

    plane_contract<T, WITH_K, VEC>(s, x, K, g, c, z, ls);
    __syncthreads();
    // x transform of the ny/2 packed rows (row pair r at offset 2 r ls); rows are the
    // fast thread index, so that neighbouring lanes read neighbouring rows rather than
    // butterflies 8 or 16 elements apart in one row (fewer shared-memory bank conflicts)
    fft_lines<T, false>(s, twx, g.ax, half, 2 * ls, 1, 0, 1, tid, nthr);
    // split each packed row into the half spectra of its two real rows.  Columns
    // kx = 0 and nx/2 of a real row are real, so one complex y transform of
    // Z = X_0 + i X_h carries both and nx/2 columns are transformed, not nx/2 + 1:
    // column 0 receives X_h as its imaginary part here (column nx/2 is rebuilt
    // after the y transform).
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5, kh = nx / 2;
    const int jr = lane % SPLIT_ROWS<T>, kg = lane / SPLIT_ROWS<T>;
    for (int r0 = warp * SPLIT_ROWS<T>; r0 < half; r0 += nw * SPLIT_ROWS<T>) {  // warp-uniform
        const int r = r0 + jr;
        const bool rok = r < half;
        C* row = s + r * 2 * ls;
        C A[SPLIT_K<T>], B[SPLIT_K<T>];
        T ah = (T)0, bh = (T)0;
#pragma unroll
        for (int t = 0; t < SPLIT_K<T>; ++t) {
            const int k = kg + SPLIT_G<T> * t;
            if (rok && k <= kh) {
                const C zk = row[posx[k]];
                const C zm = row[posx[k == 0 ? 0 : nx - k]];
                A[t] = mk<C>((zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5);
                B[t] = mk<C>((zk.y + zm.y) * (T)0.5, (zm.x - zk.x) * (T)0.5);
                if (k == kh) {
                    ah = A[t].x;
                    bh = B[t].x;
                }
            }
        }
        // X_h of both rows, from the lane holding k = nx/2 to the lane holding k = 0 (same row)
        const int src = jr + SPLIT_ROWS<T> * (kh % SPLIT_G<T>);
        ah = __shfl_sync(0xffffffffu, ah, src);
        bh = __shfl_sync(0xffffffffu, bh, src);
        __syncwarp();
#pragma unroll
        for (int t = 0; t < SPLIT_K<T>; ++t) {
            const int k = kg + SPLIT_G<T> * t;
            if (!rok) continue;
            if (k == 0) {
                row[0] = mk<C>(A[t].x, ah);
                row[ls] = mk<C>(B[t].x, bh);
            } else if (k < kh) {
                row[k] = A[t];
                row[ls + k] = B[t];
            }
        }
    }
    __syncthreads();
    fft_lines<T, false>(s, twy, g.ay, kh, 1, 1, 0, ls, tid, nthr);
    {
        // X_0(k) = (Z(k) + conj Z(-k)) / 2, X_h(k) = (Z(k) - conj Z(-k)) / 2i (one position per thread)
        C zp, zq;
        const bool act = tid < ny;
        if (act) {
            const int kk = g.fqy[tid];
            zp = s[tid * ls];
            zq = s[posy[kk == 0 ? 0 : ny - kk] * ls];
        }
        __syncthreads();
        if (act) {
            s[tid * ls] = mk<C>((zp.x + zq.x) * (T)0.5, (zp.y - zq.y) * (T)0.5);
            s[tid * ls + kh] = mk<C>((zp.y + zq.y) * (T)0.5, (zq.x - zp.x) * (T)0.5);
        }
        __syncthreads();
    }
    C* out = spec + ((long long)c * g.nz + z) * (long long)ny * nxh;
    // the plane is contiguous in both places and ny * nxh * sizeof(C) is a multiple of 16
    const int nq = ny * nxh * (int)sizeof(C) / 16;
    const float4* src4 = reinterpret_cast<const float4*>(s);
    float4* dst4 = reinterpret_cast<float4*>(out);
    for (int e = tid; e < nq; e += nthr) dst4[e] = src4[e];
}

template <typename T, bool WITH_K, bool VEC>
__global__ void __launch_bounds__(512) k_plane_fwd(const T* __restrict__ x, const T* __restrict__ K,
                                                   typename C2<T>::t* __restrict__ spec, GridDev g,
                                                   const int* __restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    plane_fwd_body<T, WITH_K, VEC>(x, K, spec, g, blockIdx.x, blockIdx.y, sm_raw);
}

// ---------------------------------------------------------------- pass 2: z transform + projection
// G_ijkl = delta_ik n_j n_l maps row i of the tensor onto row i only
// (y_ij = n_j sum_l x_il n_l), so a block takes one tensor row (components
// 3i, 3i+1, 3i+2) and W consecutive (ky, kx) columns: 3 x nz x W values,
// each row segment of W contiguous complex values read and written whole.
template <typename T> __device__ __forceinline__ T rnorm3(T a, T b, T d) { return (T)1 / sqrt(a * a + b * b + d * d); }
template <> __device__ __forceinline__ float rnorm3<float>(float a, float b, float d) {
    return rsqrtf(a * a + b * b + d * d);
}

// Shared tables of the z pass: twiddles, wave-vector components, frequencies
// of the z positions, and the block's column frequencies colk[W]
// (kx | ky << 16, -1 past the end).
template <typename T> struct ZTables {
    typename C2<T>::t* twz;
    T *qx, *qy, *qz;
    int *fqz, *colk;
};

template <typename T> __device__ __forceinline__ ZTables<T> ztables_at(unsigned char* p, const GridDev& g) {
    using C = typename C2<T>::t;
    ZTables<T> tb;
    tb.twz = reinterpret_cast<C*>(p);
    tb.qx = reinterpret_cast<T*>(tb.twz + g.nz);
    tb.qy = tb.qx + g.nxh;
    tb.qz = tb.qy + g.ny;
    tb.fqz = reinterpret_cast<int*>(tb.qz + g.nz);
    tb.colk = tb.fqz + g.nz;
    return tb;
}
template <typename T> __host__ __device__ constexpr size_t ztables_bytes(int nz, int ny, int nxh, int W) {
    return (size_t)nz * sizeof(typename C2<T>::t) + (size_t)(nxh + ny + nz) * sizeof(T) + (size_t)(nz + W) * sizeof(int);
}

template <typename T>
__device__ __forceinline__ void zproj_tables(const GridDev& g, const ProjArgs& pa, const ZTables<T>& tb) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < g.nz; i += nthr) {
        tb.twz[i] = twp<T>(g, 2)[i];
        tb.qz[i] = qtp<T>(g, pa.kind, 2)[i];
        tb.fqz[i] = g.fqz[i];
    }
    for (int i = tid; i < g.ny; i += nthr) tb.qy[i] = qtp<T>(g, pa.kind, 1)[i];
    for (int i = tid; i < g.nxh; i += nthr) tb.qx[i] = qtp<T>(g, pa.kind, 0)[i];
}

// Column frequencies of the strip starting at f0 (before the strip's first barrier).
template <typename T, int W>
__device__ __forceinline__ void zproj_columns(const GridDev& g, int f0, const ZTables<T>& tb) {
    const int nF = g.ny * g.nxh;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const int f = f0 + w;
        const int py = f / g.nxh;
        tb.colk[w] = f < nF ? (f - py * g.nxh) | (g.fqy[py] << 16) : -1;
    }
}

// The projection reaches a tensor row only through t = x_il q_l
// (y_ij = t q_j / |q|^2), and q_x, q_y are constant along a z column, so the
// z pass transforms two fields per row instead of three:
//   before the forward z transform  u = q_x x_i0 + q_y x_i1,  v = x_i2;
//   at each frequency               a = (u + q_z v) / |q|^2,  v <- q_z a;
//   after the inverse z transform   y_i0 = q_x a, y_i1 = q_y a, y_i2 = v.
// On the zero-frequency column (kx, ky) = (0, 0), where q_x = q_y = 0, the
// plane sums of x_i0 and x_i1 (real numbers) travel packed as
// u = x_i0 + i x_i1 instead, so the masked mean (zero frequency: the
// stress-controlled components kept, mask m) of all three components passes
// through; Nyquist planes are zeroed.
template <typename T> struct ZCol {
    T a, b;   // q_x(kx), q_y(ky)
    bool dc;  // (kx, ky) = (0, 0)
};
template <typename T> __device__ __forceinline__ ZCol<T> zcol(int ck, const ZTables<T>& tb) {
    ZCol<T> c{(T)0, (T)0, false};
    if (ck >= 0) {
        const int kx = ck & 0xffff, ky = ck >> 16;
        c.a = tb.qx[kx];
        c.b = tb.qy[ky];
        c.dc = kx == 0 && ky == 0;
    }
    return c;
}
template <typename T>
__device__ __forceinline__ typename C2<T>::t zpack(typename C2<T>::t v0, typename C2<T>::t v1, const ZCol<T>& c) {
    using C = typename C2<T>::t;
    if (c.dc) return mk<C>(v0.x, v1.x);
    return mk<C>(fma(c.a, v0.x, c.b * v1.x), fma(c.a, v0.y, c.b * v1.y));
}
template <typename T>
__device__ __forceinline__ void zunpack(typename C2<T>::t a, const ZCol<T>& c, typename C2<T>::t& y0,
                                        typename C2<T>::t& y1) {
    using C = typename C2<T>::t;
    if (c.dc) {
        y0 = mk<C>(a.x, (T)0);
        y1 = mk<C>(a.y, (T)0);
    } else {
        y0 = cscale(a, c.a);
        y1 = cscale(a, c.b);
    }
}
template <typename T>
__device__ __forceinline__ void zrow_proj(typename C2<T>::t& u, typename C2<T>::t& v, int kx, int ky, int kz, int nx,
                                          int ny, int nz, T m0, T m1, T m2, const ZTables<T>& tb) {
    using C = typename C2<T>::t;
    if (kx == nx / 2 || ky == ny / 2 || kz == nz / 2) {
        u = v = mk<C>((T)0, (T)0);
    } else if (kx == 0 && ky == 0) {
        if (kz == 0) {
            u = mk<C>(u.x * m0, u.y * m1);
            v = cscale(v, m2);
        } else {
            u = mk<C>((T)0, (T)0);  // q along z: y_i2 = x_i2, y_i0 = y_i1 = 0
        }
    } else {
        const T a = tb.qx[kx], b = tb.qy[ky], d = tb.qz[kz];
        const T r = (T)1 / fma(a, a, fma(b, b, d * d));
        const C t = mk<C>(fma(d, v.x, u.x) * r, fma(d, v.y, u.y) * r);
        u = t;
        v = cscale(t, d);
    }
}

// Forward z transform, projection and inverse z transform of one loaded strip
// s = [3][nz][W] (tensor row `row`): the row packed into u (slot 0) and
// v (slot 2), both transformed, projected, transformed back and unpacked into
// the three slots; ends with a barrier.
template <typename T, int W>
__device__ __forceinline__ void zproj_strip(typename C2<T>::t* s, const GridDev& g, const ProjArgs& pa, int row,
                                            const ZTables<T>& tb) {
    using C = typename C2<T>::t;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int e = tid; e < nz * W; e += nthr) s[e] = zpack<T>(s[e], s[nz * W + e], zcol<T>(tb.colk[e % W], tb));
    __syncthreads();
    fft_lines<T, false>(s, tb.twz, g.az, W, 1, 2, 2 * nz * W, W, tid, nthr);
    const T m0 = (T)pa.mask[3 * row], m1 = (T)pa.mask[3 * row + 1], m2 = (T)pa.mask[3 * row + 2];
    for (int e = tid; e < nz * W; e += nthr) {
        const int w = e % W, pz = e / W;
        const int ck = tb.colk[w];
        if (ck < 0) continue;
        const int kx = ck & 0xffff, ky = ck >> 16, kz = tb.fqz[pz];
        C* p0 = s + pz * W + w;
        C u = p0[0], v = p0[2 * nz * W];
        zrow_proj<T>(u, v, kx, ky, kz, nx, ny, nz, m0, m1, m2, tb);
        p0[0] = u;
        p0[2 * nz * W] = v;
    }
    __syncthreads();
    fft_lines<T, true>(s, tb.twz, g.az, W, 1, 2, 2 * nz * W, W, tid, nthr);
    for (int e = tid; e < nz * W; e += nthr) zunpack<T>(s[e], zcol<T>(tb.colk[e % W], tb), s[e], s[nz * W + e]);
    __syncthreads();
}

// z transform, projection and inverse z transform of one strip for the
// two-stage plans nz = 16 x 8 and 8 x 8, with one butterfly's values held in
// registers across a stage: the forward radix-R1 stage (the row packed into
// u, v on its loads); then per (column, sub) the forward radix-8 stage of u
// and v, the projection of the eight frequencies sub + R1 q it produced, and
// the inverse radix-8 stage, without leaving registers; then the inverse
// radix-R1 stage (unpacked on its stores).  The same operations in the same
// order as zproj_strip (bit-identical), with four passes over shared memory
// and four barriers fewer.  Ends with a barrier.
template <typename T, int R1, int W>
__device__ __forceinline__ void zstrip2(typename C2<T>::t* s, const GridDev& g, const ProjArgs& pa, int row,
                                        const ZTables<T>& tb) {
    using C = typename C2<T>::t;
    constexpr int R2 = 8, nz = R1 * R2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // forward radix R1 over positions j + R2 n1 of u (slot 0) and v (slot 2), twiddles after
    for (int t = tid; t < 2 * R2 * W; t += nthr) {
        const int w = t % W, jc = t / W, j = jc % R2, comp = jc / R2;  // comp warp-uniform (R2 W % 32 == 0)
        C* b = s + (2 * comp * nz + j) * W + w;
        C v[R1];
        if (comp == 0) {
            const ZCol<T> c = zcol<T>(tb.colk[w], tb);
#pragma unroll
            for (int q = 0; q < R1; ++q) v[q] = zpack<T>(b[q * R2 * W], b[(nz + q * R2) * W], c);
        } else {
#pragma unroll
            for (int q = 0; q < R1; ++q) v[q] = b[q * R2 * W];
        }
        Bfly<R1, false, C>::run(v);
        if (j) {
#pragma unroll
            for (int p = 1; p < R1; ++p) v[p] = cmul(v[p], tb.twz[p * j]);
        }
#pragma unroll
        for (int q = 0; q < R1; ++q) b[q * R2 * W] = v[q];
    }
    __syncthreads();
    const int nx = g.nx, ny = g.ny;
    const T m0 = (T)pa.mask[3 * row], m1 = (T)pa.mask[3 * row + 1], m2 = (T)pa.mask[3 * row + 2];
    for (int t = tid; t < R1 * W; t += nthr) {
        const int w = t % W, sub = t / W;
        const int ck = tb.colk[w];
        C* b = s + sub * R2 * W + w;
        C u[R2], v[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) {
            u[q] = b[q * W];
            v[q] = b[(2 * nz + q) * W];
        }
        Bfly<R2, false, C>::run(u);
        Bfly<R2, false, C>::run(v);
        if (ck >= 0) {
            const int kx = ck & 0xffff, ky = ck >> 16;
#pragma unroll
            for (int q = 0; q < R2; ++q)
                zrow_proj<T>(u[q], v[q], kx, ky, tb.fqz[sub * R2 + q], nx, ny, nz, m0, m1, m2, tb);
        }
        Bfly<R2, true, C>::run(u);
        Bfly<R2, true, C>::run(v);
#pragma unroll
        for (int q = 0; q < R2; ++q) {
            b[q * W] = u[q];
            b[(2 * nz + q) * W] = v[q];
        }
    }
    __syncthreads();
    // inverse radix R1, conjugate twiddles before; u unpacked into slots 0 and 1
    for (int t = tid; t < 2 * R2 * W; t += nthr) {
        const int w = t % W, jc = t / W, j = jc % R2, comp = jc / R2;
        C* b = s + (2 * comp * nz + j) * W + w;
        C v[R1];
#pragma unroll
        for (int q = 0; q < R1; ++q) v[q] = b[q * R2 * W];
        if (j) {
#pragma unroll
            for (int p = 1; p < R1; ++p) v[p] = cmulc(v[p], tb.twz[p * j]);
        }
        Bfly<R1, true, C>::run(v);
        if (comp == 0) {
            const ZCol<T> c = zcol<T>(tb.colk[w], tb);
#pragma unroll
            for (int q = 0; q < R1; ++q) zunpack<T>(v[q], c, b[q * R2 * W], b[(nz + q * R2) * W]);
        } else {
#pragma unroll
            for (int q = 0; q < R1; ++q) b[q * R2 * W] = v[q];
        }
    }
    __syncthreads();
}

template <typename T, int W>
__device__ __forceinline__ void zproj_body(typename C2<T>::t* __restrict__ spec, const GridDev& g,
                                           const ProjArgs& pa, const int blk, unsigned char* sm_raw) {
    using C = typename C2<T>::t;
    const int nz = g.nz;
    C* s = reinterpret_cast<C*>(sm_raw);  // [3][nz][W]
    const ZTables<T> tb = ztables_at<T>(reinterpret_cast<unsigned char*>(s + 3 * nz * W), g);
    const int tid = threadIdx.x, nthr = blockDim.x;
    // spectrum indices fit in 32 bits (9 nz ny nxh < 2^31 for axes <= MAXN)
    const int nF = g.ny * g.nxh;
    const int row = blk % 3;
    const int f0 = (blk / 3) * W;
    C* base = spec + 3 * row * nz * nF;  // component 3 row, z = 0
    zproj_tables<T>(g, pa, tb);
    zproj_columns<T, W>(g, f0, tb);
    for (int e = tid; e < 3 * nz * W; e += nthr) {
        const int w = e % W, cz = e / W;  // cz = (component within the row) * nz + z
        const int f = f0 + w;
        s[e] = f < nF ? base[cz * nF + f] : mk<C>((T)0, (T)0);
    }
    __syncthreads();
    zproj_strip<T, W>(s, g, pa, row, tb);
    for (int e = tid; e < 3 * nz * W; e += nthr) {
        const int w = e % W, cz = e / W;
        const int f = f0 + w;
        if (f < nF) base[cz * nF + f] = s[e];
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(256) k_zproj(typename C2<T>::t* __restrict__ spec, GridDev g, ProjArgs pa,
                                              const int* __restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    zproj_body<T, W>(spec, g, pa, blockIdx.x, sm_raw);
}

// ---------------------------------------------------------------- small-strain variant: symmetric projection
// Compatible small strains are sym(q (x) u).  The orthogonal projection of a
// tensor A onto them at a frequency with unit (scaled) wave vector n is
//   y = n (x) a + a (x) n - (n . a) n (x) n,   a = sym(A) n,
// which couples all nine components: a block takes the 9 components of W
// consecutive (ky, kx) columns, [9][nz][W] in shared memory.
template <typename T> constexpr int zsym_width() { return sizeof(T) == 8 ? 4 : 8; }
template <typename T> size_t zsym_smem(const GridDev& g) {
    constexpr int W = zsym_width<T>();
    return (size_t)9 * g.nz * W * sizeof(typename C2<T>::t) + ztables_bytes<T>(g.nz, g.ny, g.nxh, W) + 16;
}

template <typename T, int W>
__global__ void __launch_bounds__(256) k_zproj_sym(typename C2<T>::t* __restrict__ spec, GridDev g, ProjArgs pa,
                                                  const int* __restrict__ skip) {
    using C = typename C2<T>::t;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nz = g.nz, nx = g.nx, ny = g.ny;
    C* s = reinterpret_cast<C*>(sm_raw);  // [9][nz][W]
    const ZTables<T> tb = ztables_at<T>(reinterpret_cast<unsigned char*>(s + 9 * nz * W), g);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nF = ny * g.nxh;
    const int f0 = blockIdx.x * W;
    zproj_tables<T>(g, pa, tb);
    zproj_columns<T, W>(g, f0, tb);
    for (int e = tid; e < 9 * nz * W; e += nthr) {
        const int w = e % W, cz = e / W;  // cz = component * nz + z
        const int f = f0 + w;
        s[e] = f < nF ? spec[(long long)cz * nF + f] : mk<C>((T)0, (T)0);
    }
    __syncthreads();
    fft_lines<T, false>(s, tb.twz, g.az, W, 1, 9, nz * W, W, tid, nthr);
    for (int e = tid; e < nz * W; e += nthr) {
        const int w = e % W, pz = e / W;
        const int ck = tb.colk[w];
        if (ck < 0) continue;
        const int kx = ck & 0xffff, ky = ck >> 16, kz = tb.fqz[pz];
        C* p0 = s + pz * W + w;
        C v[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) v[c] = p0[c * nz * W];
        if (kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = cscale(v[c], (T)pa.mask[c]);
        } else if (kx == nx / 2 || ky == ny / 2 || kz == nz / 2) {
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = mk<C>((T)0, (T)0);
        } else {
            const T qa = tb.qx[kx], qb = tb.qy[ky], qd = tb.qz[kz];
            const T inv = rnorm3(qa, qb, qd);
            const T n[3] = {qa * inv, qb * inv, qd * inv};
            C a[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {  // a_j = sym(A)_jk n_k
                T re = (T)0, im = (T)0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    re += (T)0.5 * (v[3 * j + k].x + v[3 * k + j].x) * n[k];
                    im += (T)0.5 * (v[3 * j + k].y + v[3 * k + j].y) * n[k];
                }
                a[j] = mk<C>(re, im);
            }
            const C na = mk<C>(n[0] * a[0].x + n[1] * a[1].x + n[2] * a[2].x,
                               n[0] * a[0].y + n[1] * a[1].y + n[2] * a[2].y);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    v[3 * i + j] = mk<C>(n[i] * a[j].x + a[i].x * n[j] - na.x * n[i] * n[j],
                                         n[i] * a[j].y + a[i].y * n[j] - na.y * n[i] * n[j]);
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) p0[c * nz * W] = v[c];
    }
    __syncthreads();
    fft_lines<T, true>(s, tb.twz, g.az, W, 1, 9, nz * W, W, tid, nthr);
    for (int e = tid; e < 9 * nz * W; e += nthr) {
        const int w = e % W, cz = e / W;
        const int f = f0 + w;
        if (f < nF) spec[(long long)cz * nF + f] = s[e];
    }
}

// Persistent z pass on the tensor-memory accelerator: the half spectrum seen as
// a 3-D tensor [9 components][nz][ny nxh columns] (64-bit elements), a strip
// (3 components of one tensor row, all z, W columns) is one TMA box whose
// shared-memory image is exactly the [3][nz][W] layout the transforms use.
// Blocks walk the strips with two buffers: the next strip's load and the
// previous strip's store run while the current strip is transformed.  Waits
// on the load barrier are bounded (timeout -> *err = 1, GFF_ERR_TIMEOUT).
template <typename T, int W> __host__ __device__ constexpr size_t zstrip_bytes(int nz) {
    return (((size_t)3 * nz * W * sizeof(typename C2<T>::t)) + 127) / 128 * 128;
}
template <typename T, int W> size_t ztma_smem(const GridDev& g) {
    // + 127 bytes of alignment, 7 of barrier padding, 16 of barriers
    return 2 * zstrip_bytes<T, W>(g.nz) + ztables_bytes<T>(g.nz, g.ny, g.nxh, W) + 160;
}

// R1 = 0: any nz (zproj_strip), up to BT = 512 threads; R1 = 16 / 8: nz = 128 / 64 with
// the register-staged strip (zstrip2), whose fused middle stage holds 16 complex values
// (u and v of one radix-8 butterfly): BT = 256 threads, two blocks per SM in FP32 and one
// in FP64 (whose pipe, not the warps in flight, sets the pace; a cap of 128 registers
// spills), or (FP32) BT = 384, one block per SM
template <typename T, int W, int R1, int BT> constexpr int ztma_min_blocks() {
    return (R1 && sizeof(T) == 4 && BT == 256) ? 2 : 1;
}

template <typename T, int W, int R1, int BT>
__global__ void __launch_bounds__(BT, ztma_min_blocks<T, W, R1, BT>())
    k_zproj_tma(const __grid_constant__ CUtensorMap tm, GridDev g, ProjArgs pa, const int* __restrict__ skip,
                int* __restrict__ err) {
    using C = typename C2<T>::t;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    unsigned char* p = sm_raw + ((128u - (smem_addr(sm_raw) & 127u)) & 127u);  // 128-byte aligned boxes
    const size_t sb = zstrip_bytes<T, W>(g.nz);
    C* buf[2] = {reinterpret_cast<C*>(p), reinterpret_cast<C*>(p + sb)};
    const ZTables<T> tb = ztables_at<T>(p + 2 * sb, g);
    uint64_t* bar = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(tb.colk + W) + 7) & ~uintptr_t(7));
    constexpr int K = (int)(sizeof(C) / 8);  // 64-bit elements per complex value
    const uint32_t bytes = (uint32_t)(3 * g.nz * W * sizeof(C));
    const int nF = g.ny * g.nxh, total = 3 * ((nF + W - 1) / W);
    zproj_tables<T>(g, pa, tb);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    int s = blockIdx.x;
    if (threadIdx.x == 0 && s < total) tma_load_3d(buf[0], &tm, (s / 3) * W * K, 0, 3 * (s % 3), &bar[0], bytes);
    uint32_t phase[2] = {0u, 0u};
    int cur = 0;
    for (; s < total; s += gridDim.x) {
        const int nxt = s + gridDim.x;
        if (threadIdx.x == 0 && nxt < total) {
            bulk_wait_read_all();  // the other buffer's store (previous strip) has left shared memory
            tma_load_3d(buf[cur ^ 1], &tm, (nxt / 3) * W * K, 0, 3 * (nxt % 3), &bar[cur ^ 1], bytes);
        }
        zproj_columns<T, W>(g, (s / 3) * W, tb);
        const bool ok = mbar_wait(&bar[cur], phase[cur], g.wait_cycles);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[cur], phase[cur], BULK_WAIT_CYCLES);
                if (nxt < total) mbar_wait(&bar[cur ^ 1], phase[cur ^ 1], BULK_WAIT_CYCLES);
                bulk_wait_all();
            }
            __syncthreads();
            return;
        }
        phase[cur] ^= 1u;
        if constexpr (R1 > 0)
            zstrip2<T, R1, W>(buf[cur], g, pa, s % 3, tb);
        else
            zproj_strip<T, W>(buf[cur], g, pa, s % 3, tb);
        fence_proxy_async_smem();  // the transforms' writes, before the asynchronous store reads them
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tm, (s / 3) * W * K, 0, 3 * (s % 3), buf[cur]);
            bulk_commit();
        }
        cur ^= 1;
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

// ---------------------------------------------------------------- pass 3: inverse 2D transform + epilogue
// Inverse y transform, merge of the packed rows, complex-to-real x transform
// and epilogue of one plane already in shared memory s (tables loaded).
template <typename T, bool VEC>
__device__ __forceinline__ void plane_inv_compute(typename C2<T>::t* s, T* __restrict__ y, const GridDev& g,
                                                  const OutArgs& oa, const int c, const int z,
                                                  const typename C2<T>::t* twx, const typename C2<T>::t* twy,
                                                  const int* posx) {
    using C = typename C2<T>::t;
    const int nx = g.nx, ny = g.ny, nxh = g.nxh, ls = nxh, half = ny / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long N = g.N;
    const long long pl = (long long)z * ny * nx;
    const int kh0 = nx / 2;
    // columns kx = 0 and nx/2 transform back to real columns: one complex transform of X_0 + i X_h
    for (int yy = tid; yy < ny; yy += nthr) {
        const C a = s[yy * ls], b = s[yy * ls + kh0];
        s[yy * ls] = mk<C>(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    fft_lines<T, true>(s, twy, g.ay, kh0, 1, 1, 0, ls, tid, nthr);
    // merge the half spectra of rows 2r, 2r+1 into one packed complex row
    // Z_k = A_k + i B_k over all k (Hermitian symmetry of real rows), in the
    // digit-reversed order the inverse x pass expects; the real column nx/2
    // is the imaginary part of column 0 after the y transform
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5, kh = nx / 2;
    const int jr = lane % SPLIT_ROWS<T>, kg = lane / SPLIT_ROWS<T>;
    for (int r0 = warp * SPLIT_ROWS<T>; r0 < half; r0 += nw * SPLIT_ROWS<T>) {  // warp-uniform
        const int r = r0 + jr;
        const bool rok = r < half;
        C* row = s + r * 2 * ls;
        C A[SPLIT_K<T>], B[SPLIT_K<T>];
#pragma unroll
        for (int t = 0; t < SPLIT_K<T>; ++t) {
            const int k = kg + SPLIT_G<T> * t;
            if (rok && k < kh) {
                A[t] = row[k];
                B[t] = row[ls + k];
            } else if (rok && k == kh) {
                A[t] = mk<C>(row[0].y, (T)0);
                B[t] = mk<C>(row[ls].y, (T)0);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < SPLIT_K<T>; ++t) {
            const int k = kg + SPLIT_G<T> * t;
            if (rok && k <= kh) {
                if (k == 0 || k == kh) {
                    row[posx[k]] = mk<C>(A[t].x, B[t].x);
                } else {
                    row[posx[k]] = mk<C>(A[t].x - B[t].y, A[t].y + B[t].x);
                    row[posx[nx - k]] = mk<C>(A[t].x + B[t].y, B[t].x - A[t].y);
                }
            }
        }
    }
    __syncthreads();
    fft_lines<T, true>(s, twx, g.ax, half, 2 * ls, 1, 0, 1, tid, nthr);  // rows fastest, as in pass 1
    const T sc = (T)oa.scale, ad = (T)oa.add[c];
    T* yc = y + c * N;
    if (VEC) {
        // the mirror of the load in pass 1: lanes 2i, 2i+1 each read VW/2 whole
        // complex values (16 bytes) of packed row r, swap halves, and write VW
        // voxels of rows 2r (real parts) and 2r+1 (imaginary parts)
        using VT = typename V16<T>::t;
        constexpr int VW = V16<T>::n, HW = VW / 2;
        const int nxv = nx / VW, total = ny * nxv;
        const int lane = tid & 31;
        for (int e0 = tid - lane; e0 < total; e0 += nthr) {
            const int e = e0 + lane;
            const bool act = e < total;
            const int p = e & 1, q = e >> 1;
            const int r = q / nxv, xv = q - r * nxv;
            VT in;
            T* ip = reinterpret_cast<T*>(&in);
#pragma unroll
            for (int j = 0; j < VW; ++j) ip[j] = (T)0;
            if (act) in = *reinterpret_cast<const VT*>(s + r * 2 * ls + xv * VW + p * HW);
            VT o;
            T* op = reinterpret_cast<T*>(&o);
#pragma unroll
            for (int j = 0; j < HW; ++j) {
                const T recv = __shfl_xor_sync(0xffffffffu, p ? ip[2 * j] : ip[2 * j + 1], 1);
                op[j] = fma(sc, p ? recv : ip[2 * j], ad);
                op[HW + j] = fma(sc, p ? ip[2 * j + 1] : recv, ad);
            }
            if (act) *reinterpret_cast<VT*>(yc + pl + (long long)(2 * r + p) * nx + xv * VW) = o;
        }
    } else {
        for (int e = tid; e < half * nx; e += nthr) {
            const int r = e / nx, xi = e - r * nx;
            const long long v0 = pl + (long long)(2 * r) * nx + xi;
            const C zv = s[r * 2 * ls + xi];
            yc[v0] = fma(sc, zv.x, ad);
            yc[v0 + nx] = fma(sc, zv.y, ad);
        }
    }
}

// Plane (c, z) of the output set to NaN: what an inverse pass leaves where a
// bounded wait gave up, so that the failure shows in y as well as in the flag.
template <typename T>
__device__ __noinline__ void plane_fill_nan(T* y, const GridDev& g, int c, int z) {
    T* yc = y + (long long)c * g.N + (long long)z * g.ny * g.nx;
    const T nanv = (T)__int_as_float(0x7fc00000);
    for (int e = threadIdx.x; e < g.ny * g.nx; e += blockDim.x) yc[e] = nanv;
}

template <typename T>
__device__ __forceinline__ void plane_tables(const GridDev& g, typename C2<T>::t* twx, typename C2<T>::t* twy,
                                             int* posx) {
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        twx[i] = twp<T>(g, 0)[i];
        posx[i] = g.posx[i];
    }
    for (int i = threadIdx.x; i < g.ny; i += blockDim.x) twy[i] = twp<T>(g, 1)[i];
}

template <typename T, bool VEC>
__device__ __forceinline__ void plane_inv_body(const typename C2<T>::t* __restrict__ spec, T* __restrict__ y,
                                               const GridDev& g, const OutArgs& oa, const int c, const int z,
                                               unsigned char* sm_raw) {
    using C = typename C2<T>::t;
    const int nx = g.nx, ny = g.ny, nxh = g.nxh, ls = nxh;
    C* s = reinterpret_cast<C*>(sm_raw);
    C* twx = s + ny * ls;
    C* twy = twx + nx;
    int* posx = reinterpret_cast<int*>(twy + ny);
    const int tid = threadIdx.x, nthr = blockDim.x;
    plane_tables<T>(g, twx, twy, posx);
    const C* in = spec + ((long long)c * g.nz + z) * (long long)ny * nxh;
    {
        const int nq = ny * nxh * (int)sizeof(C) / 16;
        const float4* src4 = reinterpret_cast<const float4*>(in);
        float4* dst4 = reinterpret_cast<float4*>(s);
        for (int e = tid; e < nq; e += nthr) dst4[e] = __ldg(src4 + e);
    }
    __syncthreads();
    plane_inv_compute<T, VEC>(s, y, g, oa, c, z, twx, twy, posx);
}

// One block per plane (c, z) = (blockIdx.x, blockIdx.y).  The half-spectrum
// plane is one contiguous run: a single bulk asynchronous copy brings it into
// shared memory while the threads load the tables.  The wait is bounded
// (timeout -> *err = 1 when err is set, and the block leaves).
template <typename T, bool VEC>
__global__ void __launch_bounds__(512) k_plane_inv(const typename C2<T>::t* __restrict__ spec, T* __restrict__ y,
                                                   GridDev g, OutArgs oa, const int* __restrict__ skip,
                                                   int* __restrict__ err) {
    using C = typename C2<T>::t;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nx = g.nx, plane = g.ny * g.nxh;
    C* s = reinterpret_cast<C*>(sm_raw);
    C* twx = s + plane;
    C* twy = twx + nx;
    int* posx = reinterpret_cast<int*>(twy + g.ny);
    // in the ny ints after posx that only the forward pass uses (plane_smem_bytes)
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(posx + nx) + 7) & ~uintptr_t(7));
    const int c = blockIdx.x, z = blockIdx.y;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();  // the barrier is initialised before any thread waits on it
    if (threadIdx.x == 0)  // plane * sizeof(C) is a multiple of 16 (ny even), the plane start too
        bulk_load(s, spec + ((long long)c * g.nz + z) * plane, (uint32_t)(plane * sizeof(C)), bar);
    plane_tables<T>(g, twx, twy, posx);
    const bool ok = mbar_wait(bar, 0u, g.wait_cycles);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            if (err) atomicExch(err, 1);
            mbar_wait(bar, 0u, BULK_WAIT_CYCLES);  // let the copy land (bounded) before leaving
        }
        plane_fill_nan<T>(y, g, c, z);  // the plane is not computed: make that visible in y
        __syncthreads();
        return;
    }
    plane_inv_compute<T, VEC>(s, y, g, oa, c, z, twx, twy, posx);
}

// Persistent variant: each block walks the planes p = blockIdx.x + k gridDim.x
// (p = c nz + z) with two plane buffers; while one plane is transformed, the
// next arrives by a bulk asynchronous copy (the half-spectrum plane is one
// contiguous run), so the loads overlap the shared-memory FFT work.
template <typename T> size_t plane_stream_smem(const GridDev& g) {
    using C = typename C2<T>::t;
    return 2 * (size_t)g.ny * g.nxh * sizeof(C) + (size_t)(g.nx + g.ny) * sizeof(C) + g.nx * sizeof(int) + 32;
}

// up to 1024 threads in FP32; FP64 would spill at that register budget
template <typename T> constexpr int inv_stream_max_threads() { return sizeof(T) == 4 ? 1024 : 512; }

template <typename T, bool VEC>
__global__ void __launch_bounds__(inv_stream_max_threads<T>()) k_plane_inv_stream(const typename C2<T>::t* __restrict__ spec,
                                                          T* __restrict__ y, GridDev g, OutArgs oa,
                                                          const int* __restrict__ skip, int* __restrict__ err) {
    using C = typename C2<T>::t;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nx = g.nx, ny = g.ny, plane = ny * g.nxh;
    const uint32_t bytes = (uint32_t)(plane * sizeof(C));  // multiple of 16 (ny even)
    C* buf[2] = {reinterpret_cast<C*>(sm_raw), reinterpret_cast<C*>(sm_raw) + plane};
    C* twx = buf[1] + plane;
    C* twy = twx + nx;
    int* posx = reinterpret_cast<int*>(twy + ny);
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(posx + nx) + 7) & ~uintptr_t(7));
    const int total = 9 * g.nz;
    plane_tables<T>(g, twx, twy, posx);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    int p = blockIdx.x;
    if (threadIdx.x == 0 && p < total) bulk_load(buf[0], spec + (long long)p * plane, bytes, &bar[0]);
    uint32_t phase[2] = {0u, 0u};
    int cur = 0;
    for (; p < total; p += gridDim.x) {
        const int nextp = p + gridDim.x;
        if (threadIdx.x == 0 && nextp < total) {
            fence_proxy_async_smem();  // the other buffer's last readers finished at the barrier below
            bulk_load(buf[cur ^ 1], spec + (long long)nextp * plane, bytes, &bar[cur ^ 1]);
        }
        const bool ok = mbar_wait(&bar[cur], phase[cur], g.wait_cycles);
        if (__syncthreads_or(!ok)) {
            // record, let the copies in flight land (bounded), mark the planes this
            // block still owns as not computed (NaN), leave
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[cur], phase[cur], BULK_WAIT_CYCLES);
                if (nextp < total) mbar_wait(&bar[cur ^ 1], phase[cur ^ 1], BULK_WAIT_CYCLES);
            }
            for (int q = p; q < total; q += gridDim.x) plane_fill_nan<T>(y, g, q / g.nz, q % g.nz);
            __syncthreads();
            return;
        }
        phase[cur] ^= 1u;
        plane_inv_compute<T, VEC>(buf[cur], y, g, oa, p / g.nz, p % g.nz, twx, twy, posx);
        __syncthreads();
        cur ^= 1;
    }
}

// ---------------------------------------------------------------- pass 3 for two-stage plans, register-staged
// For planes with nx = ny = n = R1 R2 and the two-stage plans 16 x 8 (n = 128)
// and 8 x 8 (n = 64): the operations of plane_inv_compute in the same order
// (bit-identical results) with half its passes over shared memory.  Each
// thread keeps one butterfly's values in registers across a stage:
//   Y1  radix R2 of the inverse y transform over contiguous positions (columns
//       kx < n/2; column 0 takes X_0 + i X_h, the DC and Nyquist columns);
//   Y2  radix R1 with twiddles over stride R2, natural y order;
//   X1  merge and radix R2 of the x transform: a thread takes the butterflies
//       sub and R1 - sub (0 and R1/2) of one packed row r, whose inputs
//       Z_k = A_k + i B_k and Z_{n-k} = conj(A_k) + i conj(B_k) (A, B the half
//       spectra of rows 2r, 2r+1) come from the same stored columns; the
//       result overwrites rows 2r, 2r+1, XOR-swizzled inside each run of 8;
//   X2  radix R1 with twiddles (from a [j][p] table padded to R1 + 1 per row),
//       epilogue, stores straight to y.
// Shared memory serves 8-byte accesses a half-warp and 16-byte ones a quarter-
// warp at a time; the row pairs that share such a phase in X1 / X2 are S = L/2
// apart (L lanes per row pair), which with the row stride n/2 + 1 puts every
// access of the four phases in distinct banks.  The half-spectrum plane
// arrives by one bulk asynchronous copy with a bounded wait, as in k_plane_inv.
template <int R1, int R2> struct Inv2Plan {
    static_assert(R2 == 8 && (R1 == 8 || R1 == 16), "two-stage plans 8 x 8 and 16 x 8");
    static constexpr int n = R1 * R2, h = n / 2, nxh = h + 1;
    static constexpr int L1 = R1 / 2, G1 = 32 / L1, S1 = L1 / 2;  // X1: lanes per row pair, pairs per warp, spacing
    static constexpr int L2 = R2, G2 = 32 / R2, S2 = L2 / 2;      // X2
    static constexpr bool SAMEWARP = (G1 == G2 && S1 == S2);      // X1 and X2 give a warp the same row pairs
    static constexpr int TWS = R1 + 1;                            // row stride of the X2 twiddle table
};

__device__ __forceinline__ int swz8(int p) { return (p & ~7) | ((p ^ (p >> 3)) & 7); }
// row pair of lane group k of warp group wg: groups S apart, S G consecutive pairs per S warp groups
__device__ __forceinline__ int inv2_pair(int wg, int k, int G, int S) { return wg % S + S * k + (wg / S) * S * G; }

template <typename T, int R1, int R2>
__device__ __forceinline__ void inv2_x1(typename C2<T>::t* s, int wg, int lane) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, R2>;
    constexpr int HQ = R2 / 2;
    const int k = lane / P::L1, u = lane % P::L1;
    const int r = inv2_pair(wg, k, P::G1, P::S1);
    C* A = s + 2 * r * P::nxh;
    const C* B = A + P::nxh;
    const int c1 = u, c2 = u ? R1 - u : R1 / 2;
    const bool u0 = (u == 0);
    C p1[HQ], m1[HQ], p2[HQ], m2[HQ];
    C z0, zh;
#pragma unroll
    for (int q = 0; q < HQ; ++q) {
        const C a = A[c1 + R1 * q], b = B[c1 + R1 * q];
        p1[q] = mk<C>(a.x - b.y, a.y + b.x);
        m1[q] = mk<C>(a.x + b.y, b.x - a.y);
        if (q == 0) {  // u = 0: column 0 holds (DC, Nyquist) of both rows
            z0 = mk<C>(a.x, b.x);
            zh = mk<C>(a.y, b.y);
        }
        const C a2 = A[c2 + R1 * q], b2 = B[c2 + R1 * q];
        p2[q] = mk<C>(a2.x - b2.y, a2.y + b2.x);
        m2[q] = mk<C>(a2.x + b2.y, b2.x - a2.y);
    }
    // position sub R2 + q holds frequency k = sub + R1 q; k > n/2 reads the
    // stored column n - k: (c2 + R1 (R2-1-q)) for sub = c1 != 0, (R1 (R2-q)) for sub = 0
    C za[R2], zb[R2];
#pragma unroll
    for (int q = 0; q < HQ; ++q) {
        za[q] = (q == 0 && u0) ? z0 : p1[q];
        zb[q] = p2[q];
    }
    za[HQ] = u0 ? zh : m2[HQ - 1];
#pragma unroll
    for (int q = HQ + 1; q < R2; ++q) za[q] = u0 ? m1[R2 - q] : m2[R2 - 1 - q];
#pragma unroll
    for (int q = HQ; q < R2; ++q) zb[q] = u0 ? m2[R2 - 1 - q] : m1[R2 - 1 - q];
    Bfly<R2, true, C>::run(za);
    Bfly<R2, true, C>::run(zb);
    __syncwarp();  // every lane of the warp has read its rows before any is overwritten
#pragma unroll
    for (int q = 0; q < R2; ++q) {
        A[swz8(c1 * R2 + q)] = za[q];
        A[swz8(c2 * R2 + q)] = zb[q];
    }
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void inv2_x2(const typename C2<T>::t* s, const typename C2<T>::t* twx2, T* __restrict__ yp,
                                        T sc, T ad, int wg, int lane) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, R2>;
    const int k = lane / P::L2, j = lane % P::L2;
    const int r = inv2_pair(wg, k, P::G2, P::S2);
    const C* Z = s + 2 * r * P::nxh;
    const C* tw = twx2 + j * P::TWS;  // tw[p] = W_n^(p j)
    C v[R1];
#pragma unroll
    for (int q = 0; q < R1; ++q) v[q] = Z[swz8(j + R2 * q)];
    if (j) {
#pragma unroll
        for (int p = 1; p < R1; ++p) v[p] = cmulc(v[p], tw[p]);
    }
    Bfly<R1, true, C>::run(v);
    T* y0 = yp + (long long)(2 * r) * P::n;
#pragma unroll
    for (int q = 0; q < R1; ++q) {
        y0[j + R2 * q] = fma(sc, v[q].x, ad);
        y0[P::n + j + R2 * q] = fma(sc, v[q].y, ad);
    }
}

// blocks per SM the register budget is set for: FP32 planes of 68 KB fit three
// to an SM (256 threads at <= 85 registers) or two (512 threads at <= 64)
template <typename T, int BT> constexpr int inv2_min_blocks() { return sizeof(T) == 4 ? (BT == 256 ? 3 : 2) : 1; }

// Y1 .. X2 of one plane already in shared memory s (twiddle tables loaded); writes plane (c, z) of y.
template <typename T, int R1, int R2>
__device__ __forceinline__ void inv2_compute(typename C2<T>::t* s, const typename C2<T>::t* twy,
                                             const typename C2<T>::t* twx2, T* __restrict__ y, const GridDev& g,
                                             const OutArgs& oa, const int c, const int z) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, R2>;
    constexpr int n = P::n, h = P::h, nxh = P::nxh;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // Y1: radix R2 over positions sub R2 + q of column col
    for (int t = tid; t < h * R1; t += nthr) {
        const int col = t % h, sub = t / h;
        C* b = s + sub * R2 * nxh + col;
        C v[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) v[q] = b[q * nxh];
        if (col == 0) {
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                const C w = b[q * nxh + h];
                v[q] = mk<C>(v[q].x - w.y, v[q].y + w.x);
            }
        }
        Bfly<R2, true, C>::run(v);
#pragma unroll
        for (int q = 0; q < R2; ++q) b[q * nxh] = v[q];
    }
    __syncthreads();
    // Y2: twiddles, radix R1 over positions j + R2 q
    for (int t = tid; t < h * R2; t += nthr) {
        const int col = t % h, j = t / h;
        C* b = s + j * nxh + col;
        C v[R1];
#pragma unroll
        for (int q = 0; q < R1; ++q) v[q] = b[q * R2 * nxh];
        if (j) {
#pragma unroll
            for (int p = 1; p < R1; ++p) v[p] = cmulc(v[p], twy[p * j]);
        }
        Bfly<R1, true, C>::run(v);
#pragma unroll
        for (int q = 0; q < R1; ++q) b[q * R2 * nxh] = v[q];
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const T sc = (T)oa.scale, ad = (T)oa.add[c];
    T* yp = y + c * g.N + (long long)z * n * n;
    if (P::SAMEWARP) {
        for (int wg = warp; wg < h / P::G1; wg += nw) {  // warp-uniform
            inv2_x1<T, R1, R2>(s, wg, lane);
            __syncwarp();
            inv2_x2<T, R1, R2>(s, twx2, yp, sc, ad, wg, lane);
        }
    } else {
        for (int wg = warp; wg < h / P::G1; wg += nw) inv2_x1<T, R1, R2>(s, wg, lane);
        __syncthreads();
        for (int wg = warp; wg < h / P::G2; wg += nw) inv2_x2<T, R1, R2>(s, twx2, yp, sc, ad, wg, lane);
    }}

template <typename T, int R1, int R2, int BT>
__global__ void __launch_bounds__(BT, inv2_min_blocks<T, BT>()) k_plane_inv2(const typename C2<T>::t* __restrict__ spec,
                                                                      T* __restrict__ y, GridDev g, OutArgs oa,
                                                                      const int* __restrict__ skip,
                                                                      int* __restrict__ err) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, R2>;
    constexpr int n = P::n, nxh = P::nxh;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* s = reinterpret_cast<C*>(sm_raw);  // [n][nxh]
    C* twy = s + n * nxh;                  // [n]: W_n^k of the y axis
    C* twx2 = twy + n;                     // [R2][R1 + 1]: W_n^(p j) of the x axis
    uint64_t* bar =
        reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(twx2 + R2 * P::TWS) + 7) & ~uintptr_t(7));
    const int c = blockIdx.x, z = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0)  // n nxh sizeof(C) is a multiple of 16 (n even), the plane start too
        bulk_load(s, spec + ((long long)c * g.nz + z) * (n * nxh), (uint32_t)(n * nxh * sizeof(C)), bar);
    for (int i = tid; i < n; i += nthr) twy[i] = twp<T>(g, 1)[i];
    for (int i = tid; i < R2 * P::TWS; i += nthr) {
        const int j = i / P::TWS, p = i - j * P::TWS;
        twx2[i] = p < R1 ? twp<T>(g, 0)[p * j] : mk<C>((T)0, (T)0);
    }
    const bool ok = mbar_wait(bar, 0u, g.wait_cycles);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            if (err) atomicExch(err, 1);
            mbar_wait(bar, 0u, BULK_WAIT_CYCLES);  // let the copy land (bounded) before leaving
        }
        plane_fill_nan<T>(y, g, c, z);
        __syncthreads();
        return;
    }
    inv2_compute<T, R1, R2>(s, twy, twx2, y, g, oa, c, z);
}

// Persistent FP32 variant: each block walks the planes p = blockIdx.x + k gridDim.x
// (p = c nz + z) with two plane buffers; the next plane arrives by a bulk copy
// while the current one is transformed (two 68.6 KB planes: one block per SM).
template <typename T, int R1, int BT>
__global__ void __launch_bounds__(BT, 1) k_plane_inv2s(const typename C2<T>::t* __restrict__ spec,
                                                       T* __restrict__ y, GridDev g, OutArgs oa,
                                                       const int* __restrict__ skip, int* __restrict__ err) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, 8>;
    constexpr int n = P::n, nxh = P::nxh, plane = n * nxh;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* buf[2] = {reinterpret_cast<C*>(sm_raw), reinterpret_cast<C*>(sm_raw) + plane};
    C* twy = buf[1] + plane;
    C* twx2 = twy + n;
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(twx2 + 8 * P::TWS) + 7) & ~uintptr_t(7));
    const uint32_t bytes = (uint32_t)(plane * sizeof(C));  // a multiple of 16 (n even)
    const int total = 9 * g.nz, tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < n; i += nthr) twy[i] = twp<T>(g, 1)[i];
    for (int i = tid; i < 8 * P::TWS; i += nthr) {
        const int j = i / P::TWS, q = i - j * P::TWS;
        twx2[i] = q < R1 ? twp<T>(g, 0)[q * j] : mk<C>((T)0, (T)0);
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    int p = blockIdx.x;
    if (tid == 0 && p < total) bulk_load(buf[0], spec + (long long)p * plane, bytes, &bar[0]);
    uint32_t phase[2] = {0u, 0u};
    int cur = 0;
    for (; p < total; p += gridDim.x) {
        const int nextp = p + gridDim.x;
        if (tid == 0 && nextp < total) {
            fence_proxy_async_smem();  // the other buffer's last readers and writers finished at the barrier below
            bulk_load(buf[cur ^ 1], spec + (long long)nextp * plane, bytes, &bar[cur ^ 1]);
        }
        const bool ok = mbar_wait(&bar[cur], phase[cur], g.wait_cycles);
        if (__syncthreads_or(!ok)) {
            // record, let the copies in flight land (bounded), mark the planes this block
            // still owns as not computed (NaN), leave
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[cur], phase[cur], BULK_WAIT_CYCLES);
                if (nextp < total) mbar_wait(&bar[cur ^ 1], phase[cur ^ 1], BULK_WAIT_CYCLES);
            }
            for (int q = p; q < total; q += gridDim.x) plane_fill_nan<T>(y, g, q / g.nz, q % g.nz);
            __syncthreads();
            return;
        }
        phase[cur] ^= 1u;
        inv2_compute<T, R1, 8>(buf[cur], twy, twx2, y, g, oa, p / g.nz, p % g.nz);
        __syncthreads();
        cur ^= 1;
    }
}

template <typename T> size_t inv2s_smem(const GridDev& g) {
    using C = typename C2<T>::t;
    return (2 * (size_t)g.nx * (g.nx / 2 + 1) + (size_t)g.nx + 8 * 17) * sizeof(C) + 32;
}

template <typename T> size_t inv2_smem(const GridDev& g) {
    using C = typename C2<T>::t;
    // plane, y twiddles, x twiddle table [8][R1 + 1] (R1 <= 16), barrier
    return ((size_t)g.nx * (g.nx / 2 + 1) + (size_t)g.nx + 8 * 17) * sizeof(C) + 16;
}

// 16 x 8 -> 16, 8 x 8 -> 8; 0 if the grid has no register-staged inverse pass
int inv2_radix(const GridDev& g) {
    if (g.nx != g.ny || g.ax.nst != 2 || g.ay.nst != 2 || g.ax.radix[1] != 8 || g.ay.radix[1] != 8) return 0;
    if (g.ax.radix[0] != g.ay.radix[0]) return 0;
    return (g.ax.radix[0] == 16 || g.ax.radix[0] == 8) ? g.ax.radix[0] : 0;
}

// ---------------------------------------------------------------- pass 1 for two-stage plans, register-staged
// The mirror of k_plane_inv2 for the forward pass of planes with nx = ny = n =
// R1 8 (16 x 8, 8 x 8) with K: the operations of plane_fwd_body in the same
// order (bit-identical), with 8 passes over shared memory instead of 12:
//   C   (K:x)_c into packed rows, as in plane_fwd_body (16-byte loads);
//   X1  the thread of (packed row r, j) runs the x transform's radix-R1 stage
//       with twiddles over positions j + 8 n1 and writes positions j + 8 p
//       (XOR-swizzled inside each run of 8) in place;
//   X2  radix 8 over the runs sub and R1 - sub (0 and R1/2) of one packed row,
//       whose outputs are the mirror frequencies k and n - k, so the split into
//       the half spectra A_k, B_k of rows 2r, 2r+1 (and the packing of X_h into
//       column 0) happens in registers; written in place as rows 2r, 2r+1;
//   Y1  radix R1 of the y transform with twiddles over columns kx < n/2;
//   Y2  radix 8, stored straight to the half spectrum, except column 0, whose
//       DC and Nyquist parts are separated after one more barrier.
// (Forming K:x in registers at the X1 positions, scalar loads 8 voxels apart,
// measured 1.3x slower in FP32 at 128^3 than these 16-byte loads.)
template <typename T, int R1>
__device__ __forceinline__ void fwd2_x1(typename C2<T>::t* s, const typename C2<T>::t* twx2, int wg, int lane) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, 8>;
    const int k = lane / P::L2, j = lane % P::L2;
    const int r = inv2_pair(wg, k, P::G2, P::S2);
    C* Z = s + 2 * r * P::nxh;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = Z[j + 8 * n1];
    Bfly<R1, false, C>::run(v);
    if (j) {
        const C* tw = twx2 + j * P::TWS;
#pragma unroll
        for (int p = 1; p < R1; ++p) v[p] = cmul(v[p], tw[p]);
    }
    __syncwarp();  // every lane of the warp has read its packed row before it is overwritten
#pragma unroll
    for (int p = 0; p < R1; ++p) Z[swz8(j + 8 * p)] = v[p];
}

template <typename T, int R1>
__device__ __forceinline__ void fwd2_x2(typename C2<T>::t* s, int wg, int lane) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, 8>;
    constexpr int R2 = 8, HQ = 4, n = P::n;
    const int k = lane / P::L1, u = lane % P::L1;
    const int r = inv2_pair(wg, k, P::G1, P::S1);
    C* A = s + 2 * r * P::nxh;  // row 2r; row 2r + 1 follows at A + nxh
    const int c1 = u, c2 = u ? R1 - u : R1 / 2;
    C za[R2], zb[R2];
#pragma unroll
    for (int q = 0; q < R2; ++q) {
        za[q] = A[swz8(c1 * R2 + q)];
        zb[q] = A[swz8(c2 * R2 + q)];
    }
    Bfly<R2, false, C>::run(za);
    Bfly<R2, false, C>::run(zb);
    // za[q] holds frequency c1 + R1 q, zb[q] frequency c2 + R1 q; the mirror n - k of
    // c1 + R1 q is c2 + R1 (R2-1-q) for c1 != 0 and R1 (R2 - q) for c1 = 0
    __syncwarp();  // every lane of the warp has read its packed row before the rows are written
    const T hf = (T)0.5;
    auto split = [&](const C zk, const C zm, int kk) {
        A[kk] = mk<C>((zk.x + zm.x) * hf, (zk.y - zm.y) * hf);
        A[P::nxh + kk] = mk<C>((zk.y + zm.y) * hf, (zm.x - zk.x) * hf);
    };
    if (u) {
#pragma unroll
        for (int q = 0; q < HQ; ++q) {
            split(za[q], zb[R2 - 1 - q], c1 + R1 * q);
            split(zb[q], za[R2 - 1 - q], c2 + R1 * q);
        }
    } else {
        // k = 0 and n/2 (za[0], za[HQ]) are their own mirrors: A_0, B_0, A_h, B_h are real,
        // and column 0 carries X_0 + i X_h of both rows
        const C z0 = za[0], zh = za[HQ];
        A[0] = mk<C>((z0.x + z0.x) * hf, (zh.x + zh.x) * hf);
        A[P::nxh] = mk<C>((z0.y + z0.y) * hf, (zh.y + zh.y) * hf);
#pragma unroll
        for (int q = 1; q < HQ; ++q) split(za[q], za[R2 - q], R1 * q);
#pragma unroll
        for (int q = 0; q < HQ; ++q) split(zb[q], zb[R2 - 1 - q], c2 + R1 * q);
    }
    (void)n;
}

template <typename T, int BT> constexpr int fwd2_min_blocks() { return sizeof(T) == 4 ? (BT == 256 ? 3 : 2) : 1; }

template <typename T, int R1, int BT>
__global__ void __launch_bounds__(BT, fwd2_min_blocks<T, BT>()) k_plane_fwd2(const T* __restrict__ x,
                                                                           const T* __restrict__ K,
                                                                           typename C2<T>::t* __restrict__ spec,
                                                                           GridDev g, const int* __restrict__ skip) {
    using C = typename C2<T>::t;
    using P = Inv2Plan<R1, 8>;
    constexpr int n = P::n, h = P::h, nxh = P::nxh, R2 = 8;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* s = reinterpret_cast<C*>(sm_raw);  // [n][nxh]
    C* twy = s + n * nxh;                  // [n]: W_n^k of the y axis
    C* twx2 = twy + n;                     // [8][R1 + 1]: W_n^(p j) of the x axis
    const int c = blockIdx.x, z = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < n; i += nthr) twy[i] = twp<T>(g, 1)[i];
    for (int i = tid; i < R2 * P::TWS; i += nthr) {
        const int j = i / P::TWS, p = i - j * P::TWS;
        twx2[i] = p < R1 ? twp<T>(g, 0)[p * j] : mk<C>((T)0, (T)0);
    }
    plane_contract<T, true, true>(s, x, K, g, c, z, nxh);
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    if (P::SAMEWARP) {
        for (int wg = warp; wg < h / P::G2; wg += nw) {  // warp-uniform
            fwd2_x1<T, R1>(s, twx2, wg, lane);
            __syncwarp();
            fwd2_x2<T, R1>(s, wg, lane);
        }
    } else {
        for (int wg = warp; wg < h / P::G2; wg += nw) fwd2_x1<T, R1>(s, twx2, wg, lane);
        __syncthreads();
        for (int wg = warp; wg < h / P::G1; wg += nw) fwd2_x2<T, R1>(s, wg, lane);
    }
    __syncthreads();
    // Y1: radix R1 over positions j + 8 n1 of column col, twiddles after
    for (int t = tid; t < h * R2; t += nthr) {
        const int col = t % h, j = t / h;
        C* b = s + j * nxh + col;
        C v[R1];
#pragma unroll
        for (int q = 0; q < R1; ++q) v[q] = b[q * R2 * nxh];
        Bfly<R1, false, C>::run(v);
        if (j) {
#pragma unroll
            for (int p = 1; p < R1; ++p) v[p] = cmul(v[p], twy[p * j]);
        }
#pragma unroll
        for (int q = 0; q < R1; ++q) b[q * R2 * nxh] = v[q];
    }
    __syncthreads();
    // Y2: radix 8 over positions sub 8 + q; position sub 8 + q holds y frequency sub + R1 q
    C* out = spec + ((long long)c * g.nz + z) * (long long)n * nxh;
    for (int t = tid; t < h * R1; t += nthr) {
        const int col = t % h, sub = t / h;
        C* b = s + sub * R2 * nxh + col;
        C v[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) v[q] = b[q * nxh];
        Bfly<R2, false, C>::run(v);
        if (col == 0) {
#pragma unroll
            for (int q = 0; q < R2; ++q) b[q * nxh] = v[q];
        } else {
            C* o = out + sub * R2 * nxh + col;
#pragma unroll
            for (int q = 0; q < R2; ++q) o[q * nxh] = v[q];
        }
    }
    __syncthreads();
    // column 0 carries Z = X_0 + i X_h: X_0(k) = (Z(k) + conj Z(-k)) / 2, X_h(k) = (Z(k) - conj Z(-k)) / 2i
    for (int p = tid; p < n; p += nthr) {
        const int kk = p / R2 + R1 * (p % R2);
        const int km = kk == 0 ? 0 : n - kk;
        const C zp = s[p * nxh], zq = s[((km % R1) * R2 + km / R1) * nxh];
        out[p * nxh] = mk<C>((zp.x + zq.x) * (T)0.5, (zp.y - zq.y) * (T)0.5);
        out[p * nxh + h] = mk<C>((zp.y + zq.y) * (T)0.5, (zq.x - zp.x) * (T)0.5);
    }
}

template <typename T> size_t fwd2_smem(const GridDev& g) {
    using C = typename C2<T>::t;
    return ((size_t)g.nx * (g.nx / 2 + 1) + (size_t)g.nx + 8 * 17) * sizeof(C);
}

template <typename T> constexpr int zproj_width() { return sizeof(T) == 8 ? 8 : 16; }

template <typename T> size_t zproj_smem(const GridDev& g, int W = zproj_width<T>()) {
    using C = typename C2<T>::t;
    return (size_t)3 * g.nz * W * sizeof(C) + ztables_bytes<T>(g.nz, g.ny, g.nxh, W) + 16;
}

constexpr size_t SMEM_MAX = 227 * 1024;

// 16-byte vector access needs nx to hold whole vectors and 16-byte aligned bases
// (N is a multiple of 4 because nx and ny are even, so component offsets keep the alignment)
template <typename T> bool vec_ok(const GridDev& g, const void* p) {
    return (g.nx % (16 / (int)sizeof(T))) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

template <typename K> void allow_smem(K kern, size_t bytes) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool make_axis_plan(int n, AxisPlan& p) {
    if (n < 4 || n > MAXN || (n & 1)) return false;
    int m = n, a2 = 0, a3 = 0, a5 = 0;
    while (m % 2 == 0) { m /= 2; ++a2; }
    while (m % 3 == 0) { m /= 3; ++a3; }
    while (m % 5 == 0) { m /= 5; ++a5; }
    if (m != 1) return false;
    p.n = n;
    p.nst = 0;
    // two stages where fft2_lines has the pair
    static const int pairs[8][2] = {{16, 8}, {8, 8}, {16, 5}, {16, 3}, {8, 5}, {8, 4}, {8, 3}, {4, 4}};
    for (const auto& pr : pairs)
        if (pr[0] * pr[1] == n) {
            p.nst = 2;
            p.radix[0] = pr[0];
            p.radix[1] = pr[1];
            return true;
        }
    while (a2 >= 4) { p.radix[p.nst++] = 16; a2 -= 4; }
    if (a2 == 3) p.radix[p.nst++] = 8;
    if (a2 == 2) p.radix[p.nst++] = 4;
    if (a2 == 1) p.radix[p.nst++] = 2;
    for (int i = 0; i < a5; ++i) p.radix[p.nst++] = 5;
    for (int i = 0; i < a3; ++i) p.radix[p.nst++] = 3;
    return p.nst <= MAXST;
}

int axis_freq_of_pos(int pos, const AxisPlan& p) {
    int f = 0, mult = 1, len = p.n;
    for (int i = 0; i < p.nst; ++i) {
        const int m = len / p.radix[i];
        const int d = pos / m;
        pos -= d * m;
        f += d * mult;
        mult *= p.radix[i];
        len = m;
    }
    return f;
}

size_t plane_smem_bytes(int nx, int ny, int elem) {
    return (size_t)ny * (nx / 2 + 1) * elem + (size_t)(nx + ny) * elem + (size_t)(nx + ny) * sizeof(int) + 16;
}

namespace {

template <typename T>
cudaError_t launch_fwd(const GridDev& g, int threads, const T* x, const T* K, typename C2<T>::t* spec,
                       const int* skip, cudaStream_t st, bool vin, int planes = 0) {
    // planes > 0: that many z-planes from the ones x, K and spec point at (a chunk of the grid)
    const int nzl = planes > 0 ? planes : g.nz;
    if (threads < 0 && !(K && vin)) threads = -threads;  // projection alone, unaligned: the generic pass
    if (threads < 0) {  // register-staged pass of the two-stage plans (nx = ny = 64 or 128), -threads threads
        const size_t sm = fwd2_smem<T>(g);
        const dim3 grid(9, nzl);
        const int r1 = inv2_radix(g);
#define GFF_FWD2(R, BT)                                                             \
    if (r1 == R && threads == -BT) {                                                \
        allow_smem(k_plane_fwd2<T, R, BT>, sm);                                     \
        k_plane_fwd2<T, R, BT><<<grid, BT, sm, st>>>(x, K, spec, g, skip);          \
        return cudaGetLastError();                                                  \
    }
        GFF_FWD2(16, 256)
        GFF_FWD2(16, 512)
        GFF_FWD2(8, 256)
        GFF_FWD2(8, 512)
#undef GFF_FWD2
        return cudaErrorInvalidValue;
    }
    const size_t smA = plane_smem_bytes(g.nx, g.ny, sizeof(typename C2<T>::t));
    const dim3 gridA(9, nzl);
    if (K) {
        if (vin) {
            allow_smem(k_plane_fwd<T, true, true>, smA);
            k_plane_fwd<T, true, true><<<gridA, threads, smA, st>>>(x, K, spec, g, skip);
        } else {
            allow_smem(k_plane_fwd<T, true, false>, smA);
            k_plane_fwd<T, true, false><<<gridA, threads, smA, st>>>(x, K, spec, g, skip);
        }
    } else {
        if (vin) {
            allow_smem(k_plane_fwd<T, false, true>, smA);
            k_plane_fwd<T, false, true><<<gridA, threads, smA, st>>>(x, nullptr, spec, g, skip);
        } else {
            allow_smem(k_plane_fwd<T, false, false>, smA);
            k_plane_fwd<T, false, false><<<gridA, threads, smA, st>>>(x, nullptr, spec, g, skip);
        }
    }
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_z_w(const GridDev& g, int threads, typename C2<T>::t* spec, const ProjArgs& pa, const int* skip,
                       cudaStream_t st) {
    const size_t smB = zproj_smem<T>(g, W);
    allow_smem(k_zproj<T, W>, smB);
    k_zproj<T, W><<<zproj_blocks(g, W), threads, smB, st>>>(spec, g, pa, skip);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_z(const GridDev& g, int W, int threads, typename C2<T>::t* spec, const ProjArgs& pa,
                     const int* skip, cudaStream_t st) {
    switch (W) {
        case 4: return launch_z_w<T, 4>(g, threads, spec, pa, skip, st);
        case 8: return launch_z_w<T, 8>(g, threads, spec, pa, skip, st);
        case 16: return launch_z_w<T, 16>(g, threads, spec, pa, skip, st);
        case 32: return launch_z_w<T, 32>(g, threads, spec, pa, skip, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T> int tune_index() { return sizeof(T) == 8 ? 0 : 1; }

template <typename T>
cudaError_t launch_zsym(const GridDev& g, typename C2<T>::t* spec, const ProjArgs& pa, const int* skip,
                        cudaStream_t st) {
    constexpr int W = zsym_width<T>();
    const size_t sm = zsym_smem<T>(g);
    allow_smem(k_zproj_sym<T, W>, sm);
    k_zproj_sym<T, W><<<(g.ny * g.nxh + W - 1) / W, 256, sm, st>>>(spec, g, pa, skip);
    return cudaGetLastError();
}

// ---- TMA z pass: tensor maps and launch
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <typename T> constexpr int zmap_slot(int W) { return W == 8 ? 0 : (W == 16 ? 1 : -1); }

// The handle's half spectrum as [9][nz][ny nxh] 64-bit elements, box (W k, nz, 3); null if unavailable.
template <typename T>
const CUtensorMap* zmap(gff_handle* h, int W) {
    using C = typename C2<T>::t;
    const int pi = tune_index<T>(), wi = zmap_slot<T>(W);
    if (wi < 0) return nullptr;
    if (h->zmap_ok[pi][wi]) return &h->zmap[pi][wi];
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return nullptr;
    const GridDev& g = h->g;
    const cuuint64_t K = sizeof(C) / 8, nF = (cuuint64_t)g.ny * g.nxh;
    const cuuint64_t dims[3] = {nF * K, (cuuint64_t)g.nz, 9};
    const cuuint64_t strides[2] = {nF * sizeof(C), nF * g.nz * sizeof(C)};  // bytes, multiples of 16 (ny even)
    const cuuint32_t box[3] = {(cuuint32_t)(W * K), (cuuint32_t)g.nz, 3};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&h->zmap[pi][wi], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, h->d_spec, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return nullptr;
    h->zmap_ok[pi][wi] = true;
    return &h->zmap[pi][wi];
}

// 16 x 8 -> 16, 8 x 8 -> 8: the z plans with a register-staged strip; else 0
int z2_radix(const GridDev& g) {
    if (g.az.nst != 2 || g.az.radix[1] != 8) return 0;
    return (g.az.radix[0] == 16 || g.az.radix[0] == 8) ? g.az.radix[0] : 0;
}

// block threads of the TMA z pass: any up to 512 for the generic strip; 256, or 384 in FP32, for zstrip2
template <typename T> bool ztma_threads_ok(int R1, int threads) {
    if (!R1) return threads > 0 && threads <= 512;
    return threads == 256 || (sizeof(T) == 4 && threads == 384);
}

template <typename T, int W, int R1, int BT>
cudaError_t launch_z_tma_kb(gff_handle* h, int threads, int blocks, const ProjArgs& pa, const int* skip,
                            cudaStream_t st) {
    const CUtensorMap* tm = zmap<T>(h, W);
    if (!tm) return cudaErrorNotSupported;
    const size_t sm = ztma_smem<T, W>(h->g);
    allow_smem(k_zproj_tma<T, W, R1, BT>, sm);
    k_zproj_tma<T, W, R1, BT><<<blocks, threads, sm, st>>>(*tm, h->g, pa, skip, h->d_flag + 2);
    return cudaGetLastError();
}
template <typename T, int W, int R1>
cudaError_t launch_z_tma_k(gff_handle* h, int threads, int blocks, const ProjArgs& pa, const int* skip,
                           cudaStream_t st) {
    if (!ztma_threads_ok<T>(R1, threads)) return cudaErrorInvalidValue;
    if constexpr (R1 == 0) {
        return launch_z_tma_kb<T, W, 0, 512>(h, threads, blocks, pa, skip, st);
    } else {
        if constexpr (sizeof(T) == 4)
            if (threads == 384) return launch_z_tma_kb<T, W, R1, 384>(h, threads, blocks, pa, skip, st);
        return launch_z_tma_kb<T, W, R1, 256>(h, threads, blocks, pa, skip, st);
    }
}

// blocks > 0: the TMA z pass with the generic strip; < 0: with the register-staged strip, -blocks blocks
template <typename T, int W>
cudaError_t launch_z_tma_w(gff_handle* h, int threads, int blocks, const ProjArgs& pa, const int* skip,
                           cudaStream_t st) {
    if (blocks > 0) return launch_z_tma_k<T, W, 0>(h, threads, blocks, pa, skip, st);
    switch (z2_radix(h->g)) {
        case 16: return launch_z_tma_k<T, W, 16>(h, threads, -blocks, pa, skip, st);
        case 8: return launch_z_tma_k<T, W, 8>(h, threads, -blocks, pa, skip, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_z_tma(gff_handle* h, int W, int threads, int blocks, const ProjArgs& pa, const int* skip,
                         cudaStream_t st) {
    switch (W) {
        case 8: return launch_z_tma_w<T, 8>(h, threads, blocks, pa, skip, st);
        case 16: return launch_z_tma_w<T, 16>(h, threads, blocks, pa, skip, st);
        default: return cudaErrorInvalidValue;
    }
}

// blocks of a TMA z pass: all that fit at once, at most one per strip; 0 if it cannot run
template <typename T, int W, int R1, int BT>
int z_tma_blocks_kb(gff_handle* h, int threads) {
    const size_t sm = ztma_smem<T, W>(h->g);
    if (sm > SMEM_MAX || !zmap<T>(h, W)) return 0;
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    allow_smem(k_zproj_tma<T, W, R1, BT>, sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zproj_tma<T, W, R1, BT>, threads, sm) !=
            cudaSuccess ||
        per < 1)
        return 0;
    const int total = zproj_blocks(h->g, W);
    return nsm * per < total ? nsm * per : total;
}
template <typename T, int W, int R1>
int z_tma_blocks_k(gff_handle* h, int threads) {
    if (!ztma_threads_ok<T>(R1, threads)) return 0;
    if constexpr (R1 == 0) {
        return z_tma_blocks_kb<T, W, 0, 512>(h, threads);
    } else {
        if constexpr (sizeof(T) == 4)
            if (threads == 384) return z_tma_blocks_kb<T, W, R1, 384>(h, threads);
        return z_tma_blocks_kb<T, W, R1, 256>(h, threads);
    }
}
template <typename T, int W>
int z_tma_blocks_w(gff_handle* h, int threads, bool reg) {
    if (!reg) return z_tma_blocks_k<T, W, 0>(h, threads);
    switch (z2_radix(h->g)) {
        case 16: return z_tma_blocks_k<T, W, 16>(h, threads);
        case 8: return z_tma_blocks_k<T, W, 8>(h, threads);
        default: return 0;
    }
}
// > 0 blocks of the generic TMA z pass (reg false) or of the register-staged one (reg true); 0 if it cannot run
template <typename T>
int z_tma_blocks(gff_handle* h, int W, int threads, bool reg = false) {
    return W == 8 ? z_tma_blocks_w<T, 8>(h, threads, reg) : (W == 16 ? z_tma_blocks_w<T, 16>(h, threads, reg) : 0);
}

template <typename T>
cudaError_t launch_inv(const GridDev& g, int threads, int blocks, const typename C2<T>::t* spec, T* y,
                       const OutArgs& oa, const int* skip, cudaStream_t st, bool vout, int* err, int planes = 0) {
    // planes > 0 (one block per plane only): that many z-planes from the ones spec and y point at
    const int nzl = planes > 0 ? planes : g.nz;
    if (planes > 0 && blocks != 0 && blocks != -1) return cudaErrorInvalidValue;
    if (blocks < -1) {  // register-staged persistent pass, -blocks blocks
        const size_t sm = inv2s_smem<T>(g);
        const int r1 = inv2_radix(g);
#define GFF_INV2S(R, BT)                                                                   \
    if (r1 == R && threads == BT) {                                                        \
        allow_smem(k_plane_inv2s<T, R, BT>, sm);                                           \
        k_plane_inv2s<T, R, BT><<<-blocks, BT, sm, st>>>(spec, y, g, oa, skip, err);       \
        return cudaGetLastError();                                                         \
    }
        GFF_INV2S(16, 512)
        GFF_INV2S(8, 512)
        if constexpr (sizeof(T) == 4) {
            GFF_INV2S(16, 1024)
            GFF_INV2S(8, 1024)
        }
#undef GFF_INV2S
        return cudaErrorInvalidValue;
    }
    if (blocks < 0) {  // register-staged pass of the two-stage plans, one block per plane
        const size_t sm = inv2_smem<T>(g);
        const dim3 grid(9, nzl);
        const int r1 = inv2_radix(g);
#define GFF_INV2(R, BT)                                                              \
    if (r1 == R && threads == BT) {                                                  \
        allow_smem(k_plane_inv2<T, R, 8, BT>, sm);                                   \
        k_plane_inv2<T, R, 8, BT><<<grid, BT, sm, st>>>(spec, y, g, oa, skip, err);  \
        return cudaGetLastError();                                                   \
    }
        GFF_INV2(16, 256)
        GFF_INV2(16, 512)
        GFF_INV2(8, 256)
        GFF_INV2(8, 512)
#undef GFF_INV2
        return cudaErrorInvalidValue;
    }
    if (blocks > 0) {
        const size_t sm = plane_stream_smem<T>(g);
        if (vout) {
            allow_smem(k_plane_inv_stream<T, true>, sm);
            k_plane_inv_stream<T, true><<<blocks, threads, sm, st>>>(spec, y, g, oa, skip, err);
        } else {
            allow_smem(k_plane_inv_stream<T, false>, sm);
            k_plane_inv_stream<T, false><<<blocks, threads, sm, st>>>(spec, y, g, oa, skip, err);
        }
        return cudaGetLastError();
    }
    const size_t smA = plane_smem_bytes(g.nx, g.ny, sizeof(typename C2<T>::t));
    const dim3 gridA(9, nzl);
    if (vout) {
        allow_smem(k_plane_inv<T, true>, smA);
        k_plane_inv<T, true><<<gridA, threads, smA, st>>>(spec, y, g, oa, skip, err);
    } else {
        allow_smem(k_plane_inv<T, false>, smA);
        k_plane_inv<T, false><<<gridA, threads, smA, st>>>(spec, y, g, oa, skip, err);
    }
    return cudaGetLastError();
}


// fastest candidate of one kernel: run(i) launches candidate i `reps` times
template <typename F>
cudaError_t pick_fastest(int ncand, const bool* valid, int reps, cudaStream_t st, F run, int* best) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float bestms = 1e30f;
    *best = -1;
    for (int i = 0; i < ncand && e == cudaSuccess; ++i) {
        if (!valid[i]) continue;
        e = run(i);  // warm-up (also sets the shared-memory attribute)
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run(i);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < bestms) {
            bestms = ms;
            *best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

// blocks of the persistent inverse pass: all that fit on the GPU at once, at most one per plane
template <typename T>
int inv_stream_blocks(const GridDev& g, int threads, bool vout) {
    const size_t sm = plane_stream_smem<T>(g);
    if (sm > SMEM_MAX) return 0;
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e;
    if (vout) {
        allow_smem(k_plane_inv_stream<T, true>, sm);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_plane_inv_stream<T, true>, threads, sm);
    } else {
        allow_smem(k_plane_inv_stream<T, false>, sm);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_plane_inv_stream<T, false>, threads, sm);
    }
    if (e != cudaSuccess || per < 1) return 0;
    const int total = 9 * g.nz;
    return nsm * per < total ? nsm * per : total;
}

// blocks of the persistent register-staged inverse pass: all that fit at once, at most one per plane; 0 if it
// cannot run on this grid (plan, shared memory) with this many threads
template <typename T, int R1, int BT>
int inv2s_blocks_k(const GridDev& g) {
    const size_t sm = inv2s_smem<T>(g);
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    allow_smem(k_plane_inv2s<T, R1, BT>, sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_plane_inv2s<T, R1, BT>, BT, sm) != cudaSuccess ||
        per < 1)
        return 0;
    const int total = 9 * g.nz;
    return nsm * per < total ? nsm * per : total;
}
template <typename T>
int inv2s_blocks(const GridDev& g, int threads) {
    if (inv2s_smem<T>(g) > SMEM_MAX) return 0;
    const int r1 = inv2_radix(g);
    if (threads == 512) return r1 == 16 ? inv2s_blocks_k<T, 16, 512>(g) : (r1 == 8 ? inv2s_blocks_k<T, 8, 512>(g) : 0);
    if constexpr (sizeof(T) == 4)
        if (threads == 1024)
            return r1 == 16 ? inv2s_blocks_k<T, 16, 1024>(g) : (r1 == 8 ? inv2s_blocks_k<T, 8, 1024>(g) : 0);
    return 0;
}

template <typename T>
cudaError_t autotune_prec(gff_handle* h, T* x, T* y, const T* K) {
    using C = typename C2<T>::t;
    const GridDev& g = h->g;
    C* spec = reinterpret_cast<C*>(h->d_spec);
    cudaStream_t st = h->stream;
    const int reps = 3;
    Tune& tn = h->tune[tune_index<T>()];
    const bool vin = vec_ok<T>(g, x) && vec_ok<T>(g, K);
    // forward pass: 256 or 512 threads, or (two-stage plans, nx = ny) the register-staged pass (-256, -512)
    const bool f2 = inv2_radix(g) > 0 && fwd2_smem<T>(g) <= SMEM_MAX;
    const int tp[4] = {256, 512, -256, -512};
    const bool tv[4] = {true, true, f2, f2};
    int b = -1;
    cudaError_t e = pick_fastest(4, tv, reps, st, [&](int i) { return launch_fwd<T>(g, tp[i], x, K, spec, nullptr, st, vin); }, &b);
    if (e != cudaSuccess) return e;
    tn.t_fwd = tp[b];
    // z pass: one block per strip (W 4..32, 128 or 256 threads), or the persistent TMA pass (W 8, 16; 256, 512)
    // (the TMA pass also takes 192 / 384 threads; a strip of W columns has 16 W radix-16
    // butterflies at n = 128, its rows packed into two transformed fields)
    // and (nz = 64 or 128) the TMA pass with the register-staged strip (W 8, 16; 256 threads, or 384 in FP32)
    constexpr int NZC = 18;
    const int wz[NZC] = {4, 4, 8, 8, 16, 16, 32, 32, 8, 8, 16, 16, 8, 8, 16, 8, 16, 16};
    const int tz[NZC] = {128, 256, 128, 256, 128, 256, 128, 256, 256, 512, 256, 512, 192, 384, 384, 256, 256, 384};
    int zb[NZC] = {0};
    bool zv[NZC];
    for (int i = 0; i < 8; ++i) zv[i] = zproj_smem<T>(g, wz[i]) <= SMEM_MAX;
    for (int i = 8; i < 15; ++i) {
        zb[i] = z_tma_blocks<T>(h, wz[i], tz[i]);
        zv[i] = zb[i] > 0;
    }
    for (int i = 15; i < NZC; ++i) {  // negative: register-staged strip
        zb[i] = -z_tma_blocks<T>(h, wz[i], tz[i], true);
        zv[i] = zb[i] < 0;
    }
    ProjArgs pa;
    pa.kind = GFF_PROJ_CONTINUOUS;
    for (int c = 0; c < 9; ++c) pa.mask[c] = 0.f;
    e = pick_fastest(NZC, zv, reps, st, [&](int i) {
        return zb[i] != 0 ? launch_z_tma<T>(h, wz[i], tz[i], zb[i], pa, nullptr, st)
                     : launch_z<T>(g, wz[i], tz[i], spec, pa, nullptr, st);
    }, &b);
    if (e != cudaSuccess) return e;
    tn.wz = wz[b];
    tn.t_z = tz[b];
    tn.z_blocks = zb[b];
    OutArgs oa;
    oa.scale = 1.0;
    for (int c = 0; c < 9; ++c) oa.add[c] = 0.0;
    // one block per plane with 256 or 512 threads, the persistent streamed pass with 512 or 1024,
    // or (two-stage plans, nx = ny) the register-staged pass with 256 or 512, one block per plane, or
    // persistent with two plane buffers (512, or 1024 in FP32)
    const bool vout = vec_ok<T>(g, y);
    const int ti[8] = {256, 512, inv_stream_max_threads<T>() / 2, inv_stream_max_threads<T>(), 256, 512, 512, 1024};
    int ib[8] = {0, 0, inv_stream_blocks<T>(g, 512, vout), inv_stream_blocks<T>(g, 1024, vout), -1, -1,
                 -inv2s_blocks<T>(g, 512), -inv2s_blocks<T>(g, 1024)};
    const bool r2 = inv2_radix(g) > 0 && inv2_smem<T>(g) <= SMEM_MAX;
    const bool iv[8] = {true, true, ib[2] > 0, ib[3] > 0, r2, r2, ib[6] < -1, ib[7] < -1};
    int* err = h->d_flag + 2;
    e = pick_fastest(8, iv, reps, st, [&](int i) { return launch_inv<T>(g, ti[i], ib[i], spec, y, oa, nullptr, st, vout, err); }, &b);
    if (e != cudaSuccess) return e;
    tn.t_inv = ti[b];
    tn.inv_blocks = ib[b];
    return cudaSuccess;
}

}  // namespace

// Launch shapes set by the caller (gff_set_tiles): checked against what each variant supports.
template <typename T>
bool tiles_valid(gff_handle* h, const Tune& t) {
    const GridDev& g = h->g;
    const bool f2 = inv2_radix(g) > 0 && fwd2_smem<T>(g) <= SMEM_MAX;
    if (t.t_fwd != 256 && t.t_fwd != 512 && !(f2 && (t.t_fwd == -256 || t.t_fwd == -512))) return false;
    if (t.t_inv != 256 && t.t_inv != 512 && t.t_inv != 1024) return false;
    if (t.wz != 4 && t.wz != 8 && t.wz != 16 && t.wz != 32) return false;
    if (t.inv_blocks < -1) {  // persistent register-staged inverse: -inv_blocks blocks, at most the resident count
        const int mx = inv2s_blocks<T>(g, t.t_inv);
        if (mx < 2 || -t.inv_blocks > mx) return false;
    }
    if (t.inv_blocks == -1 && (inv2_radix(g) == 0 || inv2_smem<T>(g) > SMEM_MAX || (t.t_inv != 256 && t.t_inv != 512)))
        return false;
    if (t.z_blocks > 0) {
        if ((t.t_z != 192 && t.t_z != 256 && t.t_z != 384 && t.t_z != 512) || z_tma_blocks<T>(h, t.wz, t.t_z) < 1)
            return false;
    } else if (t.z_blocks < 0) {  // register-staged strip: -z_blocks blocks, at most the resident count
        const int mx = z_tma_blocks<T>(h, t.wz, t.t_z, true);
        if (mx < 1 || -t.z_blocks > mx) return false;  // (mx is 0 for thread counts zstrip2 does not take)
    } else if ((t.t_z != 128 && t.t_z != 256) || zproj_smem<T>(g, t.wz) > SMEM_MAX) {
        return false;
    }
    if (t.inv_blocks > 0) {
        if (plane_stream_smem<T>(g) > SMEM_MAX || t.t_inv > inv_stream_max_threads<T>()) return false;
    } else if (t.t_inv > 512 && t.inv_blocks >= -1) {
        return false;
    }
    return true;
}

bool set_tiles(gff_handle* h, const Tune& t64, const Tune& t32) {
    if (!tiles_valid<double>(h, t64) || !tiles_valid<float>(h, t32)) return false;
    h->tune[0] = t64;
    h->tune[1] = t32;
    h->tuned = true;
    return true;
}

cudaError_t autotune_galerkin(gff_handle* h) {
    // timings are taken at the default wait budget, whatever the handle's is
    const long long wait = h->g.wait_cycles;
    h->g.wait_cycles = BULK_WAIT_CYCLES;
    // the kernels' cost does not depend on the values: the handle's vectors serve as inputs
    cudaError_t e = cudaMemsetAsync(h->d_x, 0, 9 * h->N * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_x32, 0, 9 * h->N * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_K32, 0, 81 * h->N * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_Ap, 0, 9 * h->N * sizeof(double), h->stream);
    // K: the tangent buffer is only read (its contents do not matter for timing)
    if (e == cudaSuccess) e = autotune_prec<double>(h, h->d_x, h->d_Ap, h->d_K);
    if (e == cudaSuccess) e = autotune_prec<float>(h, h->d_x32, h->d_Ap32, h->d_K32);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) h->tuned = true;
    h->K32_valid = false;  // the FP32 tangent buffer was used as scratch
    h->g.wait_cycles = wait;
    return e;
}

// ---------------------------------------------------------------- batched launches
namespace {

__device__ __forceinline__ int find_rve(const int* __restrict__ start, int n, int b) {
    int r = 0;
    while (r + 1 < n && __ldg(start + r + 1) <= b) ++r;
    return r;
}

template <typename T, bool WITH_K, bool VEC>
__global__ void __launch_bounds__(512) k_plane_fwd_batch(const RveApply* __restrict__ rv, const int* __restrict__ start,
                                                         int n) {
    const int r = find_rve(start, n, blockIdx.x);
    const RveApply& a = rv[r];
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int local = blockIdx.x - start[r];
    plane_fwd_body<T, WITH_K, VEC>(static_cast<const T*>(a.x), static_cast<const T*>(a.K),
                                   static_cast<typename C2<T>::t*>(a.spec), a.g, local % 9, local / 9, sm_raw);
}

template <typename T, int W>
__global__ void __launch_bounds__(256) k_zproj_batch(const RveApply* __restrict__ rv, const int* __restrict__ start,
                                                    int n, ProjArgs pa) {
    const int r = find_rve(start, n, blockIdx.x);
    const RveApply& a = rv[r];
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    zproj_body<T, W>(static_cast<typename C2<T>::t*>(a.spec), a.g, pa, blockIdx.x - start[r], sm_raw);
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(512) k_plane_inv_batch(const RveApply* __restrict__ rv, const int* __restrict__ start,
                                                         int n) {
    const int r = find_rve(start, n, blockIdx.x);
    const RveApply& a = rv[r];
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int local = blockIdx.x - start[r];
    plane_inv_body<T, VEC>(static_cast<const typename C2<T>::t*>(a.spec), static_cast<T*>(a.y), a.g, a.oa,
                           local % 9, local / 9, sm_raw);
}

template <typename T, int W>
cudaError_t launch_zb(const BatchLaunch& bl, const ProjArgs& pa, cudaStream_t st) {
    allow_smem(k_zproj_batch<T, W>, bl.smem_z);
    k_zproj_batch<T, W><<<bl.blocks_z, bl.tn.t_z, bl.smem_z, st>>>(bl.rv, bl.start_z, bl.n, pa);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_galerkin_batch(const BatchLaunch& bl, const ProjArgs& pa, cudaStream_t st) {
    if (bl.withK) {
        if (bl.vin) {
            allow_smem(k_plane_fwd_batch<T, true, true>, bl.smem_plane);
            k_plane_fwd_batch<T, true, true><<<bl.blocks_plane, bl.tn.t_fwd, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
        } else {
            allow_smem(k_plane_fwd_batch<T, true, false>, bl.smem_plane);
            k_plane_fwd_batch<T, true, false><<<bl.blocks_plane, bl.tn.t_fwd, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
        }
    } else {
        if (bl.vin) {
            allow_smem(k_plane_fwd_batch<T, false, true>, bl.smem_plane);
            k_plane_fwd_batch<T, false, true><<<bl.blocks_plane, bl.tn.t_fwd, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
        } else {
            allow_smem(k_plane_fwd_batch<T, false, false>, bl.smem_plane);
            k_plane_fwd_batch<T, false, false><<<bl.blocks_plane, bl.tn.t_fwd, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (bl.tn.wz) {
        case 4: e = launch_zb<T, 4>(bl, pa, st); break;
        case 8: e = launch_zb<T, 8>(bl, pa, st); break;
        case 16: e = launch_zb<T, 16>(bl, pa, st); break;
        case 32: e = launch_zb<T, 32>(bl, pa, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (bl.vout) {
        allow_smem(k_plane_inv_batch<T, true>, bl.smem_plane);
        k_plane_inv_batch<T, true><<<bl.blocks_plane, bl.tn.t_inv, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
    } else {
        allow_smem(k_plane_inv_batch<T, false>, bl.smem_plane);
        k_plane_inv_batch<T, false><<<bl.blocks_plane, bl.tn.t_inv, bl.smem_plane, st>>>(bl.rv, bl.start_plane, bl.n);
    }
    return cudaGetLastError();
}

template cudaError_t launch_galerkin_batch<double>(const BatchLaunch&, const ProjArgs&, cudaStream_t);
template cudaError_t launch_galerkin_batch<float>(const BatchLaunch&, const ProjArgs&, cudaStream_t);

// Shared-memory bytes of the batched kernels (largest RVE) and the z-blocks of one RVE.
size_t batch_plane_smem(int nx, int ny, int elem) { return plane_smem_bytes(nx, ny, elem); }
template <typename T> size_t batch_z_smem(const GridDev& g, int W) { return zproj_smem<T>(g, W); }
template size_t batch_z_smem<double>(const GridDev&, int);
template size_t batch_z_smem<float>(const GridDev&, int);

// ev (optional): four events recorded before, between and after the kernels.
// skip (optional, device): when *skip != 0 at run time every kernel returns at once.
template <typename T>
cudaError_t launch_galerkin(const gff_handle* h, const T* x, const T* K, T* y, const ProjArgs& pa,
                            const OutArgs& oa, typename C2<T>::t* spec, cudaEvent_t* ev, const int* skip) {
    const GridDev& g = h->g;
    const Tune& tn = h->tune[tune_index<T>()];
    const bool vin = vec_ok<T>(g, x) && (!K || vec_ok<T>(g, K));
    const bool vout = vec_ok<T>(g, y);
    if (ev) cudaEventRecord(ev[0], h->stream);
    cudaError_t e = launch_fwd<T>(g, tn.t_fwd, x, K, spec, skip, h->stream, vin);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], h->stream);
    // the TMA pass addresses the handle's own spectrum through its tensor map
    if (pa.sym)
        e = launch_zsym<T>(g, spec, pa, skip, h->stream);
    else if (tn.z_blocks != 0 && static_cast<const void*>(spec) == h->d_spec)
        e = launch_z_tma<T>(const_cast<gff_handle*>(h), tn.wz, tn.t_z, tn.z_blocks, pa, skip, h->stream);
    else
        e = launch_z<T>(g, tn.wz, tn.t_z, spec, pa, skip, h->stream);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], h->stream);
    e = launch_inv<T>(g, tn.t_inv, tn.inv_blocks, spec, y, oa, skip, h->stream, vout, h->d_flag + 2);
    if (ev) cudaEventRecord(ev[3], h->stream);
    return e;
}

// The apply with host buffers, pipelined over chunks of z-planes: the forward
// plane pass of a chunk waits only for that chunk's host-to-device copy, and
// a chunk's device-to-host copy waits only for its inverse plane pass, so the
// copies (on the handle's copy stream) overlap the plane passes of the other
// chunks; the z pass needs every plane and runs between.  Same kernels on the
// same planes as launch_galerkin: bitwise the same y.  A persistent inverse
// pass is replaced by its one-block-per-plane counterpart (bitwise the same).
static cudaError_t host_pipe_ready(gff_handle* h, int nch) {
    cudaError_t e = cudaSuccess;
    if (!h->copy_stream) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    while (e == cudaSuccess && h->pipe_nev < 2 + 2 * nch) {
        e = cudaEventCreateWithFlags(&h->pipe_ev[h->pipe_nev], cudaEventDisableTiming);
        if (e == cudaSuccess) ++h->pipe_nev;
    }
    return e;
}

static int host_chunks(int nz, size_t bytes) {
    if (bytes < ((size_t)4 << 20)) return 1;
    return nz >= 16 ? 8 : nz / 2;
}

template <typename T>
cudaError_t launch_galerkin_host(gff_handle* h, const T* x_host, T* y_host, T* xd, T* yd, const T* K,
                                 const ProjArgs& pa, const OutArgs& oa, typename C2<T>::t* spec) {
    const GridDev& g = h->g;
    const Tune& tn = h->tune[tune_index<T>()];
    const size_t plane = (size_t)g.ny * g.nx, pspec = (size_t)g.ny * g.nxh;
    const size_t pitch = (size_t)g.N * sizeof(T);
    const int nch = host_chunks(g.nz, 9 * pitch);
    cudaError_t e = host_pipe_ready(h, nch);
    if (e != cudaSuccess) return e;
    cudaStream_t st = h->stream, cs = h->copy_stream;
    cudaEvent_t* ev = h->pipe_ev;  // [0] start, [1] done, [2, 2 + nch) copied in, [2 + nch, 2 + 2 nch) computed
    const bool vin = vec_ok<T>(g, xd) && vec_ok<T>(g, K);
    const bool vout = vec_ok<T>(g, yd);
    int t_inv = tn.t_inv, b_inv = tn.inv_blocks;
    if (b_inv < -1) {
        t_inv = 256;
        b_inv = -1;
    } else if (b_inv > 0) {
        t_inv = t_inv > 512 ? 512 : t_inv;
        b_inv = 0;
    }
    // the copies start after the work already queued on the handle's stream (it may still use xd, yd)
    if ((e = cudaEventRecord(ev[0], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev[0], 0)) != cudaSuccess)
        return e;
    for (int c = 0; c < nch; ++c) {
        const int z0 = c * g.nz / nch, z1 = (c + 1) * g.nz / nch;
        e = cudaMemcpy2DAsync(xd + z0 * plane, pitch, x_host + z0 * plane, pitch, (z1 - z0) * plane * sizeof(T), 9,
                              cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 + c], cs);
        if (e != cudaSuccess) return e;
    }
    for (int c = 0; c < nch; ++c) {
        const int z0 = c * g.nz / nch, z1 = (c + 1) * g.nz / nch;
        if ((e = cudaStreamWaitEvent(st, ev[2 + c], 0)) != cudaSuccess) return e;
        e = launch_fwd<T>(g, tn.t_fwd, xd + z0 * plane, K + z0 * plane, spec + z0 * pspec, nullptr, st, vin, z1 - z0);
        if (e != cudaSuccess) return e;
    }
    if (pa.sym)
        e = launch_zsym<T>(g, spec, pa, nullptr, st);
    else if (tn.z_blocks != 0 && static_cast<const void*>(spec) == h->d_spec)
        e = launch_z_tma<T>(h, tn.wz, tn.t_z, tn.z_blocks, pa, nullptr, st);
    else
        e = launch_z<T>(g, tn.wz, tn.t_z, spec, pa, nullptr, st);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < nch; ++c) {
        const int z0 = c * g.nz / nch, z1 = (c + 1) * g.nz / nch;
        e = launch_inv<T>(g, t_inv, b_inv, spec + z0 * pspec, yd + z0 * plane, oa, nullptr, st, vout, h->d_flag + 2,
                          z1 - z0);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 + nch + c], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[2 + nch + c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(y_host + z0 * plane, pitch, yd + z0 * plane, pitch, (z1 - z0) * plane * sizeof(T), 9,
                                  cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return e;
    }
    // the handle's stream resumes after the last copy
    if ((e = cudaEventRecord(ev[1], cs)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(st, ev[1], 0);
}

template cudaError_t launch_galerkin<double>(const gff_handle*, const double*, const double*, double*,
                                             const ProjArgs&, const OutArgs&, double2*, cudaEvent_t*, const int*);
template cudaError_t launch_galerkin<float>(const gff_handle*, const float*, const float*, float*, const ProjArgs&,
                                            const OutArgs&, float2*, cudaEvent_t*, const int*);
template cudaError_t launch_galerkin_host<double>(gff_handle*, const double*, double*, double*, double*,
                                                  const double*, const ProjArgs&, const OutArgs&, double2*);
template cudaError_t launch_galerkin_host<float>(gff_handle*, const float*, float*, float*, float*, const float*,
                                                 const ProjArgs&, const OutArgs&, float2*);

}  // namespace gff

// =================================================================== allocation-free projection
// gff_project_noalloc serves callers that may not allocate device memory
// themselves: code embedded in a host application whose allocator owns the
// whole device-memory budget, or loops that cannot afford the device-wide
// synchronisation a cudaMalloc/cudaFree may imply.  It runs the same three
// kernels as gff_project, but its scratch -- the half spectrum and the grid
// tables -- is the file-scope array below, which every GPU that loads the
// library holds until the process exits.  The paper has no counterpart.
namespace gff {
namespace {

constexpr long long NOALLOC_MAX_VOXELS = 32768;  // e.g. 32^3, 16 x 32 x 64, ...
// half spectrum: 9 nz ny (nx/2+1) complex values <= 9 N 3/4 for even nx >= 4
constexpr size_t NOALLOC_SPEC_BYTES = 9ull * (NOALLOC_MAX_VOXELS / 4 * 3) * sizeof(double2);

struct NoallocTables {
    double2 tw64[3][MAXN];
    float2 tw32[3][MAXN];
    int posx[MAXN], fqy[MAXN], fqz[MAXN];
    double qt64[2][3][MAXN];
    float qt32[2][3][MAXN];
};
constexpr size_t NOALLOC_TABLE_OFFSET = NOALLOC_SPEC_BYTES;
constexpr size_t NOALLOC_BYTES = NOALLOC_SPEC_BYTES + ((sizeof(NoallocTables) + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) by the first call made on it.  In host code the symbol
// itself is only a host-side stand-in and must never be passed to a kernel.
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

bool noalloc_plan(int n, AxisPlan& p) { return make_axis_plan(n, p); }

// Frequency at position pos after the in-place forward transform of plan p
// (the digits of pos in the plan's mixed radix, read in reverse order).
__device__ int noalloc_freq_dev(int pos, const AxisPlan& p) {
    int f = 0, mult = 1, len = p.n;
    for (int i = 0; i < p.nst; ++i) {
        const int m = len / p.radix[i];
        const int d = pos / m;
        pos -= d * m;
        f += d * mult;
        mult *= p.radix[i];
        len = m;
    }
    return f;
}

// The grid tables, written on the device by one block from the plans and box
// lengths passed by value: twiddles exp(-2 pi i k / n), wave-vector tables
// (continuous 2 pi kappa / L, discrete tan(pi kappa / n) n / L, 0 at Nyquist)
// and the position/frequency maps of the in-place transforms.
__global__ void k_noalloc_tables(NoallocTables* t, AxisPlan ax, AxisPlan ay, AxisPlan az, double Lx, double Ly,
                                 double Lz) {
    const AxisPlan* pl[3] = {&ax, &ay, &az};
    const double L[3] = {Lx, Ly, Lz};
    for (int a = 0; a < 3; ++a) {
        const int n = pl[a]->n;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double sn, cs;
            sincospi(2.0 * k / n, &sn, &cs);
            t->tw64[a][k] = make_double2(cs, -sn);
            t->tw32[a][k] = make_float2((float)cs, (float)-sn);
            const int kappa = (2 * k < n) ? k : k - n;
            const double qc = 2.0 * 3.141592653589793238462643383279502884 * kappa / L[a];
            const double qd = (2 * k == n) ? 0.0 : sinpi((double)kappa / n) / cospi((double)kappa / n) * n / L[a];
            t->qt64[0][a][k] = qc;
            t->qt64[1][a][k] = qd;
            t->qt32[0][a][k] = (float)qc;
            t->qt32[1][a][k] = (float)qd;
        }
    }
    for (int p = threadIdx.x; p < ax.n; p += blockDim.x) t->posx[noalloc_freq_dev(p, ax)] = p;
    for (int p = threadIdx.x; p < ay.n; p += blockDim.x) t->fqy[p] = noalloc_freq_dev(p, ay);
    for (int p = threadIdx.x; p < az.n; p += blockDim.x) t->fqz[p] = noalloc_freq_dev(p, az);
}

// Every CUDA call is checked where it is made, so that an error is reported
// by the call that caused it.
template <typename K> cudaError_t noalloc_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t noalloc_launch(const GridDev& g, const T* x, T* y, const ProjArgs& pa, const OutArgs& oa,
                           typename C2<T>::t* spec, cudaStream_t st) {
    const size_t smA = plane_smem_bytes(g.nx, g.ny, sizeof(typename C2<T>::t));
    const size_t smB = zproj_smem<T>(g);
    constexpr int W = zproj_width<T>();
    const dim3 gridA(9, g.nz);
    cudaError_t e = noalloc_smem(k_plane_fwd<T, false, false>, smA);
    if (e != cudaSuccess) return e;
    k_plane_fwd<T, false, false><<<gridA, 512, smA, st>>>(x, nullptr, spec, g, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = noalloc_smem(k_zproj<T, W>, smB)) != cudaSuccess) return e;
    k_zproj<T, W><<<zproj_blocks(g, W), 256, smB, st>>>(spec, g, pa, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = noalloc_smem(k_plane_inv<T, false>, smA)) != cudaSuccess) return e;
    // no status word: a bounded wait that gives up leaves its plane of y as NaN
    k_plane_inv<T, false><<<gridA, 512, smA, st>>>(spec, y, g, oa, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace
}  // namespace gff

// No cudaMalloc, cudaFree or other allocating call is made here; see gff.h.
__attribute__((visibility("default"))) gff_status gff_project_noalloc(const gff_grid* grid, int projection,
                                                                      int precision, const uint8_t* mask9,
                                                                      const void* x_dev, void* y_dev, void* stream) {
    using namespace gff;
    if (!grid || !x_dev || !y_dev || x_dev == y_dev) return GFF_ERR_ARG;
    if (projection != GFF_PROJ_CONTINUOUS && projection != GFF_PROJ_DISCRETE) return GFF_ERR_ARG;
    if (precision != GFF_PREC_FP64 && precision != GFF_PREC_MIXED) return GFF_ERR_ARG;
    GridDev g{};
    const int n3[3] = {grid->nx, grid->ny, grid->nz};
    AxisPlan* pl[3] = {&g.ax, &g.ay, &g.az};
    for (int a = 0; a < 3; ++a) {
        if (!noalloc_plan(n3[a], *pl[a])) return GFF_ERR_ARG;
        if (!(grid->L[a] > 0)) return GFF_ERR_ARG;
    }
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > NOALLOC_MAX_VOXELS) return GFF_ERR_ARG;  // larger grids need gff_create + gff_project

    // a CUDA error left pending by an earlier call belongs to that call: report it, do not clear it
    if (cudaPeekAtLastError() != cudaSuccess) return GFF_ERR_CUDA;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return GFF_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* d = static_cast<unsigned char*>(base);
    NoallocTables* dt = reinterpret_cast<NoallocTables*>(d + NOALLOC_TABLE_OFFSET);
    // grid tables, written on the device in stream order (no host buffer is involved)
    k_noalloc_tables<<<1, 128, 0, st>>>(dt, g.ax, g.ay, g.az, grid->L[0], grid->L[1], grid->L[2]);
    if (cudaGetLastError() != cudaSuccess) return GFF_ERR_CUDA;

    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.nxh = grid->nx / 2 + 1;
    g.N = N;
    g.wait_cycles = BULK_WAIT_CYCLES;
    for (int a = 0; a < 3; ++a) {
        g.tw64[a] = dt->tw64[a];
        g.tw32[a] = dt->tw32[a];
        for (int kind = 0; kind < 2; ++kind) {
            g.qt64[kind][a] = dt->qt64[kind][a];
            g.qt32[kind][a] = dt->qt32[kind][a];
        }
    }
    g.posx = dt->posx;
    g.fqy = dt->fqy;
    g.fqz = dt->fqz;
    ProjArgs pa;
    pa.kind = projection;
    for (int c = 0; c < 9; ++c) pa.mask[c] = (mask9 && mask9[c]) ? 1.0f : 0.0f;
    OutArgs oa;
    oa.scale = 1.0 / (double)N;
    for (int c = 0; c < 9; ++c) oa.add[c] = 0.0;
    // the spectrum is fully written by the first kernel before it is read: nothing to clear
    cudaError_t e;
    if (precision == GFF_PREC_FP64)
        e = noalloc_launch<double>(g, (const double*)x_dev, (double*)y_dev, pa, oa, reinterpret_cast<double2*>(d), st);
    else
        e = noalloc_launch<float>(g, (const float*)x_dev, (float*)y_dev, pa, oa, reinterpret_cast<float2*>(d), st);
    return e == cudaSuccess ? GFF_OK : GFF_ERR_CUDA;
}
