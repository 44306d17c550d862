// Kernels of the warm-start U-Net (3x3x3 periodic convolutions on voxel grids).
//
// Activations are bfloat16, channels-last [V][C] with a row stride (so a
// tensor can be a channel slice of a concatenation buffer); accumulation is
// FP32.  The convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16 bf16 -> f32): M = voxels (16 per warp, 64 per block),
// N = output channels (<= 64), K = 27 taps x input channels (16 per step);
// the A fragment of a tap reads the 16 voxels' periodic neighbours.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gff {
namespace unet {

using bf16 = __nv_bfloat16;

struct Dims {
    int nz, ny, nx;
    long long V;
};

// voxel v -> periodic neighbour at offset (dz, dy, dx) of tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)
__device__ __forceinline__ long long neighbour(const Dims& d, long long v, int t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const long long plane = (long long)d.ny * d.nx;
    int z = (int)(v / plane);
    long long rem = v - (long long)z * plane;
    int y = (int)(rem / d.nx);
    int x = (int)(rem - (long long)y * d.nx);
    z += dz;
    y += dy;
    x += dx;
    z = z < 0 ? z + d.nz : (z >= d.nz ? z - d.nz : z);
    y = y < 0 ? y + d.ny : (y >= d.ny ? y - d.ny : y);
    x = x < 0 ? x + d.nx : (x >= d.nx ? x - d.nx : x);
    return ((long long)z * d.ny + y) * d.nx + x;
}

// negative-side slope of the activation: plain ReLU let whole layers die in training
constexpr float LEAK = 0.125f;

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// out[v, co] = act(bias[co] + sum_{t, ci} W[t][co][ci] in[nb(v, t), ci])
// in: cin channels (multiple of 16) at stride sin; W: [27][NT*8][cin] bf16;
// out: NT*8 channels at stride sout.  RELU: leaky ReLU (slope LEAK for z <= 0).
// Block = 4 warps = 64 voxels.
template <int NT, bool RELU>
__global__ void __launch_bounds__(128) k_conv3(const bf16* __restrict__ in, int sin, int cin,
                                               const bf16* __restrict__ W, const float* __restrict__ bias,
                                               bf16* __restrict__ out, int sout, Dims d) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const long long v0 = ((long long)blockIdx.x * 4 + warp) * 16;
    if (v0 >= d.V) return;
    const long long va = v0 + g, vb = v0 + g + 8;
    const bool oka = va < d.V, okb = vb < d.V;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int cout = NT * 8;
    for (int t = 0; t < 27; ++t) {
        const long long qa = neighbour(d, oka ? va : v0, t);
        const long long qb = neighbour(d, okb ? vb : v0, t);
        const bf16* ra = in + qa * sin + 2 * tq;
        const bf16* rb = in + qb * sin + 2 * tq;
        const bf16* wt = W + (long long)t * cout * cin + (long long)g * cin + 2 * tq;
        for (int kc = 0; kc < cin; kc += 16) {
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t*>(ra + kc);
            a[1] = *reinterpret_cast<const uint32_t*>(rb + kc);
            a[2] = *reinterpret_cast<const uint32_t*>(ra + kc + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(rb + kc + 8);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                uint32_t b[2];
                const bf16* wj = wt + (long long)j * 8 * cin + kc;
                b[0] = __ldg(reinterpret_cast<const unsigned int*>(wj));
                b[1] = __ldg(reinterpret_cast<const unsigned int*>(wj + 8));
                mma_bf16(acc[j], a, b);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int co = j * 8 + 2 * tq;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
        float r0 = acc[j][0] + b0, r1 = acc[j][1] + b1, r2 = acc[j][2] + b0, r3 = acc[j][3] + b1;
        if (RELU) {
            r0 = r0 > 0.f ? r0 : LEAK * r0;
            r1 = r1 > 0.f ? r1 : LEAK * r1;
            r2 = r2 > 0.f ? r2 : LEAK * r2;
            r3 = r3 > 0.f ? r3 : LEAK * r3;
        }
        if (oka) *reinterpret_cast<__nv_bfloat162*>(out + va * sout + co) = __floats2bfloat162_rn(r0, r1);
        if (okb) *reinterpret_cast<__nv_bfloat162*>(out + vb * sout + co) = __floats2bfloat162_rn(r2, r3);
    }
}

// dz = da * (act > 0 ? 1 : LEAK), C channels (exact in bfloat16: LEAK is a power of two)
__global__ void k_relu_mask(const bf16* __restrict__ da, int sda, const bf16* __restrict__ act, int sact,
                            bf16* __restrict__ dz, int sdz, int C, long long V) {
    const long long n = V * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        const float a = __bfloat162float(act[v * sact + c]);
        dz[v * sdz + c] = a > 0.f ? da[v * sda + c] : __float2bfloat16(LEAK * __bfloat162float(da[v * sda + c]));
    }
}

// dW[t][co][ci] += sum_v dz[v, co] in[nb(v, t), ci]   (FP32, atomically over voxel chunks)
// grid (27, chunks), 256 threads, dynamic smem 64 * (cout + cin) floats.
__global__ void __launch_bounds__(256) k_wgrad(const bf16* __restrict__ in, int sin, int cin,
                                               const bf16* __restrict__ dz, int sdz, int cout,
                                               float* __restrict__ dW, Dims d, long long chunk) {
    extern __shared__ float wsm[];
    float* sdz_ = wsm;              // [64][cout]
    float* sin_ = wsm + 64 * cout;  // [64][cin]
    const int t = blockIdx.x;
    const long long vbeg = (long long)blockIdx.y * chunk;
    const long long vend = min(vbeg + chunk, d.V);
    const int npair = cout * cin;
    // this thread's (co, ci) pairs: pr = tid + 256 k (unused slots point at pair 0 and are never stored)
    float acc[32];
    int oo[32], ii[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int pr = threadIdx.x + k * 256;
        acc[k] = 0.f;
        oo[k] = pr < npair ? pr / cin : 0;
        ii[k] = pr < npair ? pr - (pr / cin) * cin : 0;
    }
    for (long long tb = vbeg; tb < vend; tb += 64) {
        const int nv = (int)min((long long)64, vend - tb);
        for (int e = threadIdx.x; e < 64 * cout; e += blockDim.x) {
            const int r = e / cout, c = e - r * cout;
            sdz_[e] = r < nv ? __bfloat162float(dz[(tb + r) * sdz + c]) : 0.f;
        }
        for (int e = threadIdx.x; e < 64 * cin; e += blockDim.x) {
            const int r = e / cin, c = e - r * cin;
            sin_[e] = r < nv ? __bfloat162float(in[neighbour(d, tb + r, t) * sin + c]) : 0.f;
        }
        __syncthreads();
        for (int r = 0; r < nv; ++r) {
            const float* dzr = sdz_ + r * cout;
            const float* inr = sin_ + r * cin;
#pragma unroll
            for (int k = 0; k < 32; ++k) acc[k] = fmaf(dzr[oo[k]], inr[ii[k]], acc[k]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int pr = threadIdx.x + k * 256;
        if (pr < npair) atomicAdd(dW + (long long)t * npair + pr, acc[k]);
    }
}

// db[c] += sum_v dz[v, c]
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ dz, int sdz, int C, long long V,
                                                   float* __restrict__ db) {
    __shared__ float part[64];
    if (threadIdx.x < 64) part[threadIdx.x] = 0.f;
    __syncthreads();
    const int c = threadIdx.x % C;
    const int rows_per = blockDim.x / C;
    float s = 0.f;
    if (threadIdx.x < rows_per * C)
        for (long long v = (long long)blockIdx.x * rows_per + threadIdx.x / C; v < V; v += (long long)gridDim.x * rows_per)
            s += __bfloat162float(dz[v * sdz + c]);
    if (threadIdx.x < rows_per * C) atomicAdd(part + c, s);
    __syncthreads();
    if (threadIdx.x < C) atomicAdd(db + threadIdx.x, part[threadIdx.x]);
}

// 2x2x2 average pooling: out (coarse dims dc) from in (fine)
__global__ void k_pool(const bf16* __restrict__ in, int sin, bf16* __restrict__ out, int sout, int C, Dims dc) {
    const long long n = dc.V * C;
    const int fx = 2 * dc.nx, fy = 2 * dc.ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        const int z = (int)(v / ((long long)dc.ny * dc.nx)), y = (int)((v / dc.nx) % dc.ny), x = (int)(v % dc.nx);
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e)
                    s += __bfloat162float(in[(((long long)(2 * z + a) * fy + 2 * y + b) * fx + 2 * x + e) * sin + c]);
        out[v * sout + c] = __float2bfloat16(s * 0.125f);
    }
}

// out[child] = in[parent] (fine dims df)
__global__ void k_up(const bf16* __restrict__ in, int sin, bf16* __restrict__ out, int sout, int C, Dims df) {
    const long long n = df.V * C;
    const int cy = df.ny / 2, cx = df.nx / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        const int z = (int)(v / ((long long)df.ny * df.nx)), y = (int)((v / df.nx) % df.ny), x = (int)(v % df.nx);
        out[v * sout + c] = in[(((long long)(z / 2) * cy + y / 2) * cx + x / 2) * sin + c];
    }
}

// gradient of nearest upsampling: din[parent] = sum of the 8 children (coarse dims dc)
__global__ void k_up_grad(const bf16* __restrict__ dout, int sdo, bf16* __restrict__ din, int sdi, int C, Dims dc) {
    const long long n = dc.V * C;
    const int fx = 2 * dc.nx, fy = 2 * dc.ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        const int z = (int)(v / ((long long)dc.ny * dc.nx)), y = (int)((v / dc.nx) % dc.ny), x = (int)(v % dc.nx);
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e)
                    s += __bfloat162float(dout[(((long long)(2 * z + a) * fy + 2 * y + b) * fx + 2 * x + e) * sdo + c]);
        din[v * sdi + c] = __float2bfloat16(s);
    }
}

// out[child] = skip[child] + dpool[parent] / 8   (fine dims df)
__global__ void k_pool_grad_add(const bf16* __restrict__ skip, int ssk, const bf16* __restrict__ dp, int sdp,
                                bf16* __restrict__ out, int sout, int C, Dims df) {
    const long long n = df.V * C;
    const int cy = df.ny / 2, cx = df.nx / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        const int z = (int)(v / ((long long)df.ny * df.nx)), y = (int)((v / df.nx) % df.ny), x = (int)(v % df.nx);
        const float s = __bfloat162float(skip[v * ssk + c]) +
                        0.125f * __bfloat162float(dp[(((long long)(z / 2) * cy + y / 2) * cx + x / 2) * sdp + c]);
        out[v * sout + c] = __float2bfloat16(s);
    }
}

// 1x1 head: y[v][o] = b[o] + sum_i Wr[o][i] a[v][i]   (Wr: bfloat16-rounded weights held in FP32)
__global__ void k_head_fwd(const bf16* __restrict__ a, int sa, const float* __restrict__ Wr, const float* __restrict__ b,
                           float* __restrict__ y, int cin, int cout, long long V) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float xi[16];
        for (int i = 0; i < cin; ++i) xi[i] = __bfloat162float(a[v * sa + i]);
        for (int o = 0; o < cout; ++o) {
            float s = b[o];
            for (int i = 0; i < cin; ++i) s = fmaf(Wr[o * cin + i], xi[i], s);
            y[v * cout + o] = s;
        }
    }
}

// head backward: da[v][i] = bf16(sum_o Wr[o][i] dy[v][o]); dW[o][i] += sum_v dy[v][o] a[v][i]; db[o] += sum_v dy[v][o]
__global__ void __launch_bounds__(256) k_head_bwd(const bf16* __restrict__ a, int sa, const float* __restrict__ Wr,
                                                  const float* __restrict__ dy, bf16* __restrict__ da, int sda,
                                                  float* __restrict__ dW, float* __restrict__ db, int cin, int cout,
                                                  long long V) {
    __shared__ float pw[16 * 16 + 16];
    for (int e = threadIdx.x; e < 16 * 16 + 16; e += blockDim.x) pw[e] = 0.f;
    __syncthreads();
    float lw[9 * 16], lb[9];
    for (int k = 0; k < cout * cin; ++k) lw[k] = 0.f;
    for (int o = 0; o < cout; ++o) lb[o] = 0.f;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float xi[16], g[9];
        for (int i = 0; i < cin; ++i) xi[i] = __bfloat162float(a[v * sa + i]);
        for (int o = 0; o < cout; ++o) {
            g[o] = dy[v * cout + o];
            lb[o] += g[o];
            for (int i = 0; i < cin; ++i) lw[o * cin + i] = fmaf(g[o], xi[i], lw[o * cin + i]);
        }
        for (int i = 0; i < cin; ++i) {
            float s = 0.f;
            for (int o = 0; o < cout; ++o) s = fmaf(Wr[o * cin + i], g[o], s);
            da[v * sda + i] = __float2bfloat16(s);
        }
    }
    for (int k = 0; k < cout * cin; ++k) atomicAdd(pw + k, lw[k]);
    for (int o = 0; o < cout; ++o) atomicAdd(pw + 256 + o, lb[o]);
    __syncthreads();
    for (int k = threadIdx.x; k < cout * cin; k += blockDim.x) atomicAdd(dW + k, pw[k]);
    for (int o = threadIdx.x; o < cout; o += blockDim.x) atomicAdd(db + o, pw[256 + o]);
}

// mean squared error: dy = 2 (y - t) / n, loss += sum (y - t)^2 / n
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                                             long long n, double* __restrict__ loss) {
    __shared__ double part[8];
    double s = 0.0;
    const double inv = 1.0 / (double)n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = (float)(2.0 * d * inv);
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        atomicAdd(loss, tot * inv);
    }
}

// out += sum_i g[i]^2
__global__ void __launch_bounds__(256) k_sumsq(const float* __restrict__ g, long long n, double* __restrict__ out) {
    __shared__ double part[8];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)g[i] * g[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        atomicAdd(out, tot);
    }
}

// Adam on the flat parameter vector (FP32 master weights); the gradient is
// scaled down to global norm `clip` when sqrt(*gn2) exceeds it
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       const double* __restrict__ gn2, float clip) {
    const double gn = sqrt(*gn2);
    const float sc = gn > clip ? (float)(clip / gn) : 1.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = sc * g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bfloat16 copies of one conv layer: forward [27][co][ci] and data-gradient [27][ci][co] with flipped taps
__global__ void k_refresh(const float* __restrict__ w, bf16* __restrict__ wf, bf16* __restrict__ wd, int cout, int cin) {
    const long long n = 27LL * cout * cin;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / ((long long)cout * cin));
        const int rem = (int)(e - (long long)t * cout * cin);
        const int o = rem / cin, i = rem - o * cin;
        const bf16 r = __float2bfloat16(w[e]);
        wf[e] = r;
        wd[((long long)(26 - t) * cin + i) * cout + o] = r;
    }
}

__global__ void k_round_f32(const float* __restrict__ w, float* __restrict__ wr, int n) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        wr[e] = __bfloat162float(__float2bfloat16(w[e]));
}

}  // namespace unet
}  // namespace gff
