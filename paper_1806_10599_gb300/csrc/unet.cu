// Learned warm start: a 4-level 3D U-Net (channels 16, 32, 64, 64) trained on
// the solver's own load increments to propose the fluctuation-strain
// increment that starts the Newton iteration (the paper leaves the initial
// guess open, Sect. 2.1; this network is not in the paper).
//
// Input per voxel (IN_CH = 32 channels): the grain's orientation quaternion
// (4) and phase (1), the prescribed macroscopic increment d_k / |d_k| (9; d
// is dFbar on strain-controlled components, 0 on stress-controlled ones),
// the previous increment's normalised fluctuation increment y_{k-1} (9) and
// its direction d_{k-1} / |d_{k-1}| (9).  Output (9): the correction c with
// y_k ~ s y_{k-1} + c, s = cos(d_k, d_{k-1}), where
// y_k = (F_k - F_{k-1} - dFbar_k) / |d_k|.  The head starts at zero, so an
// untrained network reproduces the plain extrapolation.  bfloat16 weights
// and activations, FP32 accumulation on the tensor cores (unet_kernels.cuh),
// FP32 master weights updated by Adam.  The whole network is periodic
// (wrapping 3x3x3 taps, 2x2x2 pooling, nearest upsampling), so one set of
// weights serves any cubic grid whose size is a multiple of 8.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gff_internal.cuh"
#include "unet_kernels.cuh"

using namespace gff;
using namespace gff::unet;

namespace {

struct LayerDef {
    int cin, cout;
};
// e1a e1b e2a e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b
constexpr int NL = 14;
constexpr int IN_CH = 32;
constexpr LayerDef kL[NL] = {{IN_CH, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64},  {64, 64}, {64, 64},
                             {64, 64}, {128, 64}, {64, 64}, {96, 32}, {32, 32}, {48, 16}, {16, 16}};
constexpr int HEAD_IN = 16, HEAD_OUT = 9;

inline int pad16(int c) { return (c + 15) / 16 * 16; }
constexpr float GRAD_CLIP = 1.0f;  // global gradient-norm bound of a training step

struct View {
    bf16* p;
    int s;  // row stride in elements
};

}  // namespace

struct gff_unet {
    int device = 0;
    uint64_t seed = 0;
    // parameters (padded layout): per conv layer W [27][cout][cinp] then b [cout]; head W [9][16], b [9]
    size_t off_w[NL], off_b[NL], off_hw = 0, off_hb = 0, nparam = 0;
    float* d_w = nullptr;
    float* d_g = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    bf16* d_wf = nullptr;  // forward copies, same offsets as d_w (W parts)
    bf16* d_wd = nullptr;  // data-gradient copies (flipped, transposed)
    float* d_whr = nullptr;
    int adam_t = 0;
    // activations for grid n (levels n, n/2, n/4, n/8)
    int n = 0;
    void* arena = nullptr;
    View X, Ae1a, CAT1, P1, Ae2a, CAT2, P2, Ae3a, CAT3, P3, Ae4a, E4, Ad3a, D3, Ad2a, D2, Ad1a, D1;
    View gAe1a, gCAT1, gP1, gAe2a, gCAT2, gP2, gAe3a, gCAT3, gP3, gAe4a, gE4, gAd3a, gD3, gAd2a, gD2, gAd1a, gD1,
        gE3, gE2, gE1, DZ;
    float* Y = nullptr;
    float* dY = nullptr;
    double* d_loss = nullptr;
    // training samples (grid sample_n): inputs [V][IN_CH] bf16, targets [V][9] f32
    int sample_n = 0;
    std::vector<bf16*> sx;
    std::vector<float*> sy;
    std::vector<double> se;  // mean square of each sample's target
    int sampling = 0;        // 0: shuffled epochs; 1: half uniform, half in proportion to se
    std::string err;
};

namespace {

gff_status ufail(gff_unet* u, gff_status st, const char* msg, cudaError_t e = cudaSuccess) {
    if (u) {
        u->err = msg;
        if (e != cudaSuccess) u->err += std::string(": ") + cudaGetErrorString(e);
    }
    return st;
}

#define UTRY(expr)                                                         \
    do {                                                                   \
        cudaError_t e_ = (expr);                                           \
        if (e_ != cudaSuccess) return ufail(u, GFF_ERR_CUDA, #expr, e_);   \
    } while (0)

Dims dims_of(int n, int level) {
    const int m = n >> level;
    return Dims{m, m, m, (long long)m * m * m};
}

int grid_of(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b > 2048 ? 2048 : (b < 1 ? 1 : b));
}

// SplitMix64 stream for the initial weights
uint64_t sm64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

gff_status refresh_copies(gff_unet* u, cudaStream_t st) {
    for (int l = 0; l < NL; ++l) {
        const int cinp = pad16(kL[l].cin), cout = kL[l].cout;
        k_refresh<<<grid_of(27LL * cout * cinp), 256, 0, st>>>(u->d_w + u->off_w[l], u->d_wf + u->off_w[l],
                                                             u->d_wd + u->off_w[l], cout, cinp);
    }
    k_round_f32<<<1, 256, 0, st>>>(u->d_w + u->off_hw, u->d_whr, HEAD_OUT * HEAD_IN);
    UTRY(cudaGetLastError());
    return GFF_OK;
}

gff_status ensure_buffers(gff_unet* u, int n) {
    if (u->n == n && u->arena) return GFF_OK;
    if (n < 8 || n % 8) return ufail(u, GFF_ERR_ARG, "U-Net grids need n divisible by 8");
    if (u->arena) cudaFree(u->arena);
    u->arena = nullptr;
    u->n = 0;
    long long V[4];
    for (int l = 0; l < 4; ++l) V[l] = dims_of(n, l).V;
    struct Want {
        View* v;
        int level, ch;
    };
    // forward activations and their gradients
    Want w[] = {{&u->X, 0, IN_CH},     {&u->Ae1a, 0, 16},  {&u->CAT1, 0, 48},  {&u->P1, 1, 16},    {&u->Ae2a, 1, 32},
                {&u->CAT2, 1, 96},  {&u->P2, 2, 32},    {&u->Ae3a, 2, 64},  {&u->CAT3, 2, 128}, {&u->P3, 3, 64},
                {&u->Ae4a, 3, 64},  {&u->E4, 3, 64},    {&u->Ad3a, 2, 64},  {&u->D3, 2, 64},    {&u->Ad2a, 1, 32},
                {&u->D2, 1, 32},    {&u->Ad1a, 0, 16},  {&u->D1, 0, 16},    {&u->gAe1a, 0, 16}, {&u->gCAT1, 0, 48},
                {&u->gP1, 1, 16},   {&u->gAe2a, 1, 32}, {&u->gCAT2, 1, 96}, {&u->gP2, 2, 32},   {&u->gAe3a, 2, 64},
                {&u->gCAT3, 2, 128}, {&u->gP3, 3, 64},  {&u->gAe4a, 3, 64}, {&u->gE4, 3, 64},   {&u->gAd3a, 2, 64},
                {&u->gD3, 2, 64},   {&u->gAd2a, 1, 32}, {&u->gD2, 1, 32},   {&u->gAd1a, 0, 16}, {&u->gD1, 0, 16},
                {&u->gE3, 2, 64},   {&u->gE2, 1, 32},   {&u->gE1, 0, 16},   {&u->DZ, 0, 64}};
    size_t off = 0;
    std::vector<size_t> offs;
    for (auto& x : w) {
        offs.push_back(off);
        off += ((size_t)V[x.level] * x.ch * sizeof(bf16) + 255) / 256 * 256;
    }
    const size_t oY = off;
    off += ((size_t)V[0] * HEAD_OUT * sizeof(float) + 255) / 256 * 256;
    const size_t odY = off;
    off += ((size_t)V[0] * HEAD_OUT * sizeof(float) + 255) / 256 * 256;
    const size_t oL = off;
    off += 256;
    cudaError_t e = cudaMalloc(&u->arena, off);
    if (e != cudaSuccess) return ufail(u, GFF_ERR_OOM, "U-Net activations", e);
    e = cudaMemset(u->arena, 0, off);
    if (e != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net activations", e);
    unsigned char* b = static_cast<unsigned char*>(u->arena);
    for (size_t i = 0; i < sizeof(w) / sizeof(w[0]); ++i) *w[i].v = View{reinterpret_cast<bf16*>(b + offs[i]), w[i].ch};
    u->Y = reinterpret_cast<float*>(b + oY);
    u->dY = reinterpret_cast<float*>(b + odY);
    u->d_loss = reinterpret_cast<double*>(b + oL);
    u->n = n;
    return GFF_OK;
}

View slice(View v, int c0) { return View{v.p + c0, v.s}; }

// forward conv of layer l: in (cinp channels) -> out (cout channels), leaky ReLU
cudaError_t conv_fwd(gff_unet* u, int l, View in, View out, Dims d, cudaStream_t st) {
    const int cinp = pad16(kL[l].cin), cout = kL[l].cout;
    const bf16* W = u->d_wf + u->off_w[l];
    const float* b = u->d_w + u->off_b[l];
    const int blocks = (int)((d.V + 63) / 64);
    switch (cout) {
        case 16: k_conv3<2, true><<<blocks, 128, 0, st>>>(in.p, in.s, cinp, W, b, out.p, out.s, d); break;
        case 32: k_conv3<4, true><<<blocks, 128, 0, st>>>(in.p, in.s, cinp, W, b, out.p, out.s, d); break;
        case 64: k_conv3<8, true><<<blocks, 128, 0, st>>>(in.p, in.s, cinp, W, b, out.p, out.s, d); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// data gradient of layer l: dz (cout channels) -> din (cinp channels)
cudaError_t conv_dgrad(gff_unet* u, int l, View dz, View din, Dims d, cudaStream_t st) {
    const int cinp = pad16(kL[l].cin), cout = kL[l].cout;
    const bf16* W = u->d_wd + u->off_w[l];
    const int blocks = (int)((d.V + 63) / 64);
    switch (cinp) {
        case 16: k_conv3<2, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        case 32: k_conv3<4, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        case 48: k_conv3<6, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        case 64: k_conv3<8, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        case 96: k_conv3<12, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        case 128: k_conv3<16, false><<<blocks, 128, 0, st>>>(dz.p, dz.s, cout, W, nullptr, din.p, din.s, d); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// weight and bias gradients of layer l from its input and dz
cudaError_t conv_wgrad(gff_unet* u, int l, View in, View dz, Dims d, cudaStream_t st) {
    const int cinp = pad16(kL[l].cin), cout = kL[l].cout;
    long long chunks = (d.V + 4095) / 4096;
    if (chunks < 1) chunks = 1;
    const long long chunk = (d.V + chunks - 1) / chunks;
    const size_t smem = 64 * (cout + cinp) * sizeof(float);
    k_wgrad<<<dim3(27, (unsigned)chunks), 256, smem, st>>>(in.p, in.s, cinp, dz.p, dz.s, cout, u->d_g + u->off_w[l], d,
                                                           chunk);
    k_bias_grad<<<grid_of(d.V), 256, 0, st>>>(dz.p, dz.s, cout, d.V, u->d_g + u->off_b[l]);
    return cudaGetLastError();
}

gff_status forward(gff_unet* u, View X, cudaStream_t st) {
    const Dims d0 = dims_of(u->n, 0), d1 = dims_of(u->n, 1), d2 = dims_of(u->n, 2), d3 = dims_of(u->n, 3);
    UTRY(conv_fwd(u, 0, X, u->Ae1a, d0, st));
    UTRY(conv_fwd(u, 1, u->Ae1a, slice(u->CAT1, 32), d0, st));  // e1
    k_pool<<<grid_of(d1.V * 16), 256, 0, st>>>(u->CAT1.p + 32, u->CAT1.s, u->P1.p, u->P1.s, 16, d1);
    UTRY(conv_fwd(u, 2, u->P1, u->Ae2a, d1, st));
    UTRY(conv_fwd(u, 3, u->Ae2a, slice(u->CAT2, 64), d1, st));  // e2
    k_pool<<<grid_of(d2.V * 32), 256, 0, st>>>(u->CAT2.p + 64, u->CAT2.s, u->P2.p, u->P2.s, 32, d2);
    UTRY(conv_fwd(u, 4, u->P2, u->Ae3a, d2, st));
    UTRY(conv_fwd(u, 5, u->Ae3a, slice(u->CAT3, 64), d2, st));  // e3
    k_pool<<<grid_of(d3.V * 64), 256, 0, st>>>(u->CAT3.p + 64, u->CAT3.s, u->P3.p, u->P3.s, 64, d3);
    UTRY(conv_fwd(u, 6, u->P3, u->Ae4a, d3, st));
    UTRY(conv_fwd(u, 7, u->Ae4a, u->E4, d3, st));
    k_up<<<grid_of(d2.V * 64), 256, 0, st>>>(u->E4.p, u->E4.s, u->CAT3.p, u->CAT3.s, 64, d2);
    UTRY(conv_fwd(u, 8, u->CAT3, u->Ad3a, d2, st));
    UTRY(conv_fwd(u, 9, u->Ad3a, u->D3, d2, st));
    k_up<<<grid_of(d1.V * 64), 256, 0, st>>>(u->D3.p, u->D3.s, u->CAT2.p, u->CAT2.s, 64, d1);
    UTRY(conv_fwd(u, 10, u->CAT2, u->Ad2a, d1, st));
    UTRY(conv_fwd(u, 11, u->Ad2a, u->D2, d1, st));
    k_up<<<grid_of(d0.V * 32), 256, 0, st>>>(u->D2.p, u->D2.s, u->CAT1.p, u->CAT1.s, 32, d0);
    UTRY(conv_fwd(u, 12, u->CAT1, u->Ad1a, d0, st));
    UTRY(conv_fwd(u, 13, u->Ad1a, u->D1, d0, st));
    k_head_fwd<<<grid_of(d0.V), 256, 0, st>>>(u->D1.p, u->D1.s, u->d_whr, u->d_w + u->off_hb, u->Y, HEAD_IN, HEAD_OUT,
                                             d0.V);
    UTRY(cudaGetLastError());
    return GFF_OK;
}

// one conv-activation backward: dz = da (.) (out > 0 ? 1 : LEAK); weight/bias grads; din (if wanted)
gff_status back_layer(gff_unet* u, int l, View in, View out, View da, View* din, Dims d, cudaStream_t st) {
    const int cout = kL[l].cout;
    View dz{u->DZ.p, cout};
    k_relu_mask<<<grid_of(d.V * cout), 256, 0, st>>>(da.p, da.s, out.p, out.s, dz.p, dz.s, cout, d.V);
    UTRY(cudaGetLastError());
    UTRY(conv_wgrad(u, l, in, dz, d, st));
    if (din) UTRY(conv_dgrad(u, l, dz, *din, d, st));
    return GFF_OK;
}

// gradients of all parameters for the loss gradient in u->dY (forward must have run on X)
gff_status backward(gff_unet* u, View X, cudaStream_t st) {
    const Dims d0 = dims_of(u->n, 0), d1 = dims_of(u->n, 1), d2 = dims_of(u->n, 2), d3 = dims_of(u->n, 3);
    UTRY(cudaMemsetAsync(u->d_g, 0, u->nparam * sizeof(float), st));
    k_head_bwd<<<grid_of(d0.V), 256, 0, st>>>(u->D1.p, u->D1.s, u->d_whr, u->dY, u->gD1.p, u->gD1.s,
                                             u->d_g + u->off_hw, u->d_g + u->off_hb, HEAD_IN, HEAD_OUT, d0.V);
    UTRY(cudaGetLastError());
    gff_status s;
#define B_(expr) \
    if ((s = (expr)) != GFF_OK) return s
    B_(back_layer(u, 13, u->Ad1a, u->D1, u->gD1, &u->gAd1a, d0, st));
    B_(back_layer(u, 12, u->CAT1, u->Ad1a, u->gAd1a, &u->gCAT1, d0, st));
    k_up_grad<<<grid_of(d1.V * 32), 256, 0, st>>>(u->gCAT1.p, u->gCAT1.s, u->gD2.p, u->gD2.s, 32, d1);
    B_(back_layer(u, 11, u->Ad2a, u->D2, u->gD2, &u->gAd2a, d1, st));
    B_(back_layer(u, 10, u->CAT2, u->Ad2a, u->gAd2a, &u->gCAT2, d1, st));
    k_up_grad<<<grid_of(d2.V * 64), 256, 0, st>>>(u->gCAT2.p, u->gCAT2.s, u->gD3.p, u->gD3.s, 64, d2);
    B_(back_layer(u, 9, u->Ad3a, u->D3, u->gD3, &u->gAd3a, d2, st));
    B_(back_layer(u, 8, u->CAT3, u->Ad3a, u->gAd3a, &u->gCAT3, d2, st));
    k_up_grad<<<grid_of(d3.V * 64), 256, 0, st>>>(u->gCAT3.p, u->gCAT3.s, u->gE4.p, u->gE4.s, 64, d3);
    B_(back_layer(u, 7, u->Ae4a, u->E4, u->gE4, &u->gAe4a, d3, st));
    B_(back_layer(u, 6, u->P3, u->Ae4a, u->gAe4a, &u->gP3, d3, st));
    k_pool_grad_add<<<grid_of(d2.V * 64), 256, 0, st>>>(u->gCAT3.p + 64, u->gCAT3.s, u->gP3.p, u->gP3.s, u->gE3.p,
                                                        u->gE3.s, 64, d2);
    B_(back_layer(u, 5, u->Ae3a, slice(u->CAT3, 64), u->gE3, &u->gAe3a, d2, st));
    B_(back_layer(u, 4, u->P2, u->Ae3a, u->gAe3a, &u->gP2, d2, st));
    k_pool_grad_add<<<grid_of(d1.V * 32), 256, 0, st>>>(u->gCAT2.p + 64, u->gCAT2.s, u->gP2.p, u->gP2.s, u->gE2.p,
                                                        u->gE2.s, 32, d1);
    B_(back_layer(u, 3, u->Ae2a, slice(u->CAT2, 64), u->gE2, &u->gAe2a, d1, st));
    B_(back_layer(u, 2, u->P1, u->Ae2a, u->gAe2a, &u->gP1, d1, st));
    k_pool_grad_add<<<grid_of(d0.V * 16), 256, 0, st>>>(u->gCAT1.p + 32, u->gCAT1.s, u->gP1.p, u->gP1.s, u->gE1.p,
                                                        u->gE1.s, 16, d0);
    B_(back_layer(u, 1, u->Ae1a, slice(u->CAT1, 32), u->gE1, &u->gAe1a, d0, st));
    B_(back_layer(u, 0, X, u->Ae1a, u->gAe1a, nullptr, d0, st));
#undef B_
    UTRY(cudaGetLastError());
    return GFF_OK;
}

// ---------------------------------------------------------------- solver glue
__global__ void k_unet_input(const int* __restrict__ gid, const float* __restrict__ gq /* [ng][5] */, Nine9 dfn,
                             const float* __restrict__ yprev /* [9][V] or null */, Nine9 dprev,
                             bf16* __restrict__ x, long long V) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float* q = gq + 5LL * gid[v];
        bf16* r = x + v * IN_CH;
        for (int c = 0; c < 5; ++c) r[c] = __float2bfloat16(q[c]);
        for (int c = 0; c < 9; ++c) {
            r[5 + c] = __float2bfloat16((float)dfn.v[c]);
            r[14 + c] = __float2bfloat16(yprev ? yprev[c * V + v] : 0.f);
            r[23 + c] = __float2bfloat16((float)dprev.v[c]);
        }
    }
}

// target[v][c] = y[c][v] - s yprev[c][v]
__global__ void k_unet_target(const float* __restrict__ y, const float* __restrict__ yprev, float s,
                              float* __restrict__ t, long long V) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < 9; ++c) t[v * 9 + c] = y[c * V + v] - (yprev ? s * yprev[c * V + v] : 0.f);
}

// field[c][v] = scale (s yprev[c][v] + corr[v][c])   (either part may be null)
__global__ void k_guess_field(const float* __restrict__ yprev, float s, const float* __restrict__ corr, float scale,
                              float* __restrict__ f, long long V) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < 9; ++c) {
            float a = yprev ? s * yprev[c * V + v] : 0.f;
            if (corr) a += corr[v * 9 + c];
            f[c * V + v] = scale * a;
        }
}

double norm9(const double* a) {
    double s = 0.0;
    for (int c = 0; c < 9; ++c) s += a[c] * a[c];
    return std::sqrt(s);
}

// Network inputs for an increment with prescribed change d after the recorded history (yprev, dprev: may be
// absent).  Returns s = cos(d, dprev) (0 without history).
double make_input(gff_unet* u, gff_handle* h, const double* d, const float* yprev, const double* dprev, bf16* x,
                  cudaStream_t st) {
    const double nd = norm9(d), np = dprev ? norm9(dprev) : 0.0;
    Nine9 dfn, dpn;
    double s = 0.0;
    for (int c = 0; c < 9; ++c) {
        dfn.v[c] = d[c] / nd;
        dpn.v[c] = np > 0 ? dprev[c] / np : 0.0;
        s += dfn.v[c] * dpn.v[c];
    }
    (void)u;
    k_unet_input<<<grid_of(h->N), 256, 0, st>>>(h->d_gid, h->d_gq, dfn, np > 0 ? yprev : nullptr, dpn, x, h->N);
    return s;
}

}  // namespace

// ---------------------------------------------------------------- used by the solver (api.cu)
namespace gff {

// F^0 += G^(|d| (s y_{k-1} + U(x)))  (network) or G^(|d| s y_{k-1})  (u null: extrapolation)
cudaError_t warm_guess(gff_unet* u, gff_handle* h, const double* d9, int* applied) {
    *applied = 0;
    const double nrm = norm9(d9);
    if (!(nrm > 0)) return cudaSuccess;
    const bool hist = h->nhist >= 1;
    if (!u && !hist) return cudaSuccess;  // nothing to extrapolate
    cudaStream_t st = h->stream;
    const float* yprev = hist ? h->d_yhist + (size_t)h->ycur * 9 * h->N : nullptr;
    double s = 0.0;
    if (hist) {
        const double np = norm9(h->prev_d9);
        for (int c = 0; c < 9; ++c) s += d9[c] * h->prev_d9[c];
        s /= nrm * np;
    }
    const float* corr = nullptr;
    if (u) {
        if (h->grid.nx != h->grid.ny || h->grid.ny != h->grid.nz) return cudaErrorInvalidValue;
        if (ensure_buffers(u, h->grid.nx) != GFF_OK) return cudaErrorMemoryAllocation;
        make_input(u, h, d9, yprev, hist ? h->prev_d9 : nullptr, u->X.p, st);
        if (forward(u, u->X, st) != GFF_OK) return cudaErrorUnknown;
        corr = u->Y;
    }
    k_guess_field<<<grid_of(h->N), 256, 0, st>>>(yprev, (float)s, corr, (float)nrm, h->d_x32, h->N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ProjArgs pa;
    pa.kind = h->opt.projection;
    pa.sym = h->small_strain;
    for (int c = 0; c < 9; ++c) pa.mask[c] = 0.f;  // compatible, zero mean
    OutArgs oa;
    oa.scale = 1.0 / (double)h->N;
    for (int c = 0; c < 9; ++c) oa.add[c] = 0.0;
    e = launch_galerkin<float>(h, h->d_x32, (const float*)nullptr, h->d_Ap32, pa, oa, reinterpret_cast<float2*>(h->d_spec));
    if (e != cudaSuccess) return e;
    e = launch_axpy_to64<float>(h->d_Fk, h->d_Ap32, 9 * h->N, st);
    if (e == cudaSuccess) *applied = 1;
    return e;
}

}  // namespace gff

// ---------------------------------------------------------------- C ABI
#define UEXPORT __attribute__((visibility("default")))

UEXPORT gff_status gff_unet_create(uint64_t seed, gff_unet** out) {
    if (!out) return GFF_ERR_ARG;
    gff_unet* u = new gff_unet();
    *out = u;
    u->seed = seed;
    cudaGetDevice(&u->device);
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        u->off_w[l] = off;
        off += 27ULL * kL[l].cout * pad16(kL[l].cin);
        u->off_b[l] = off;
        off += kL[l].cout;
    }
    u->off_hw = off;
    off += HEAD_OUT * HEAD_IN;
    u->off_hb = off;
    off += HEAD_OUT;
    u->nparam = off;
    // He-uniform convolution weights from a SplitMix64 stream; zero biases, padding and head
    std::vector<float> w(off, 0.f);
    uint64_t s = seed;
    auto unif = [&]() { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); };
    for (int l = 0; l < NL; ++l) {
        const int ci = kL[l].cin, cip = pad16(ci), co = kL[l].cout;
        const double lim = std::sqrt(6.0 / (27.0 * ci));
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < co; ++o)
                for (int i = 0; i < ci; ++i) w[u->off_w[l] + ((size_t)t * co + o) * cip + i] = (float)((2 * unif() - 1) * lim);
    }
    // the head starts at zero: the untrained network adds nothing to the extrapolation
    cudaError_t e = cudaSuccess;
    void** bufs[] = {(void**)&u->d_w, (void**)&u->d_g, (void**)&u->d_m, (void**)&u->d_v};
    for (auto b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(b, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->d_wf, off * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc(&u->d_wd, off * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc(&u->d_whr, HEAD_OUT * HEAD_IN * sizeof(float));
    if (e != cudaSuccess) return ufail(u, GFF_ERR_OOM, "U-Net parameters", e);
    if (e == cudaSuccess) e = cudaMemcpy(u->d_w, w.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(u->d_m, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(u->d_v, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(u->d_wf, 0, off * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMemset(u->d_wd, 0, off * sizeof(bf16));
    if (e != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net parameters", e);
    gff_status st = refresh_copies(u, nullptr);
    if (st != GFF_OK) return st;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? GFF_OK : ufail(u, GFF_ERR_CUDA, "U-Net init", e);
}

UEXPORT void gff_unet_destroy(gff_unet* u) {
    if (!u) return;
    cudaFree(u->d_w);
    cudaFree(u->d_g);
    cudaFree(u->d_m);
    cudaFree(u->d_v);
    cudaFree(u->d_wf);
    cudaFree(u->d_wd);
    cudaFree(u->d_whr);
    cudaFree(u->arena);
    for (auto p : u->sx) cudaFree(p);
    for (auto p : u->sy) cudaFree(p);
    delete u;
}

UEXPORT const char* gff_unet_last_error(const gff_unet* u) { return u ? u->err.c_str() : "null network"; }

UEXPORT size_t gff_unet_num_params(const gff_unet* u) {
    size_t n = 0;
    for (int l = 0; l < NL; ++l) n += 27ULL * kL[l].cout * kL[l].cin + kL[l].cout;
    (void)u;
    return n + HEAD_OUT * HEAD_IN + HEAD_OUT;
}

// logical (unpadded) order: per layer W[27][cout][cin] then b[cout]; head W[9][16], b[9]
static gff_status copy_params(gff_unet* u, float* host, const float* src_dev) {
    std::vector<float> all(u->nparam);
    cudaError_t e = cudaMemcpy(all.data(), src_dev, u->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net params", e);
    size_t k = 0;
    for (int l = 0; l < NL; ++l) {
        const int ci = kL[l].cin, cip = pad16(ci), co = kL[l].cout;
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < co; ++o)
                for (int i = 0; i < ci; ++i) host[k++] = all[u->off_w[l] + ((size_t)t * co + o) * cip + i];
        for (int o = 0; o < co; ++o) host[k++] = all[u->off_b[l] + o];
    }
    for (int j = 0; j < HEAD_OUT * HEAD_IN + HEAD_OUT; ++j) host[k++] = all[u->off_hw + j];
    return GFF_OK;
}

UEXPORT gff_status gff_unet_get_params(gff_unet* u, float* host) {
    if (!u || !host) return GFF_ERR_ARG;
    return copy_params(u, host, u->d_w);
}

UEXPORT gff_status gff_unet_set_params(gff_unet* u, const float* host) {
    if (!u || !host) return GFF_ERR_ARG;
    std::vector<float> all(u->nparam, 0.f);
    size_t k = 0;
    for (int l = 0; l < NL; ++l) {
        const int ci = kL[l].cin, cip = pad16(ci), co = kL[l].cout;
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < co; ++o)
                for (int i = 0; i < ci; ++i) all[u->off_w[l] + ((size_t)t * co + o) * cip + i] = host[k++];
        for (int o = 0; o < co; ++o) all[u->off_b[l] + o] = host[k++];
    }
    for (int j = 0; j < HEAD_OUT * HEAD_IN + HEAD_OUT; ++j) all[u->off_hw + j] = host[k++];
    cudaError_t e = cudaMemcpy(u->d_w, all.data(), u->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net params", e);
    gff_status st = refresh_copies(u, nullptr);
    if (st != GFF_OK) return st;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? GFF_OK : ufail(u, GFF_ERR_CUDA, "U-Net params", e);
}

// Forward (and, with target, the loss and all parameter gradients) on host
// inputs: x [V][14], target [V][9] (may be NULL), y [V][9], grads in the
// order of gff_unet_get_params (may be NULL).  For tests and inspection.
UEXPORT gff_status gff_unet_eval_host(gff_unet* u, int n, const float* x, const float* target, float* y,
                                      double* loss, float* grads) {
    if (!u || !x || !y) return GFF_ERR_ARG;
    gff_status st = ensure_buffers(u, n);
    if (st != GFF_OK) return st;
    const long long V = (long long)n * n * n;
    std::vector<bf16> xb((size_t)V * IN_CH);
    for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16(x[i]);
    UTRY(cudaMemcpy(u->X.p, xb.data(), xb.size() * sizeof(bf16), cudaMemcpyHostToDevice));
    if ((st = forward(u, u->X, nullptr)) != GFF_OK) return st;
    UTRY(cudaMemcpy(y, u->Y, (size_t)V * 9 * sizeof(float), cudaMemcpyDeviceToHost));
    if (!target) return GFF_OK;
    float* dT = nullptr;
    UTRY(cudaMalloc(&dT, (size_t)V * 9 * sizeof(float)));
    cudaError_t e = cudaMemcpy(dT, target, (size_t)V * 9 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(u->d_loss, 0, sizeof(double));
    if (e == cudaSuccess) {
        k_mse<<<grid_of(V * 9), 256>>>(u->Y, dT, u->dY, V * 9, u->d_loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && (st = backward(u, u->X, nullptr)) != GFF_OK) {
        cudaFree(dT);
        return st;
    }
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, u->d_loss, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dT);
    if (e != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net eval", e);
    return grads ? copy_params(u, grads, u->d_g) : GFF_OK;
}

// Mean square of a device target of n values (for the sampling weights).
static gff_status target_energy(gff_unet* u, const float* t, long long n, double* e) {
    double* d = nullptr;
    UTRY(cudaMalloc(&d, sizeof(double)));
    cudaError_t err = cudaMemset(d, 0, sizeof(double));
    if (err == cudaSuccess) {
        k_sumsq<<<grid_of(n), 256>>>(t, n, d);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpy(e, d, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) return ufail(u, GFF_ERR_CUDA, "U-Net sample", err);
    *e /= (double)n;
    return GFF_OK;
}

// Keep the last increment of h (inputs and the fluctuation-increment target) as a training sample.
UEXPORT gff_status gff_unet_add_sample(gff_unet* u, gff_handle* h) {
    if (!u || !h) return GFF_ERR_ARG;
    if (h->nhist < 1) return ufail(u, GFF_ERR_STATE, "the handle has no completed increment with a strain increment");
    if (h->grid.nx != h->grid.ny || h->grid.ny != h->grid.nz || h->grid.nx % 8)
        return ufail(u, GFF_ERR_ARG, "samples need cubic grids with n divisible by 8");
    if (u->sample_n && u->sample_n != h->grid.nx) return ufail(u, GFF_ERR_ARG, "all samples must share one grid");
    const long long V = h->N;
    bf16* x = nullptr;
    float* t = nullptr;
    UTRY(cudaMalloc(&x, (size_t)V * IN_CH * sizeof(bf16)));
    cudaError_t e = cudaMalloc(&t, (size_t)V * 9 * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(x);
        return ufail(u, GFF_ERR_OOM, "U-Net sample", e);
    }
    // increment k = the last completed one; its predecessor k-1 is on record when nhist = 2
    const float* yk = h->d_yhist + (size_t)h->ycur * 9 * V;
    const float* ykm1 = h->nhist >= 2 ? h->d_yhist + (size_t)(h->ycur ^ 1) * 9 * V : nullptr;
    const double s = make_input(u, h, h->prev_d9, ykm1, ykm1 ? h->prev2_d9 : nullptr, x, h->stream);
    k_unet_target<<<grid_of(V), 256, 0, h->stream>>>(yk, ykm1, (float)s, t, V);
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaFree(x);
        cudaFree(t);
        return ufail(u, GFF_ERR_CUDA, "U-Net sample", e);
    }
    double en = 0.0;
    gff_status se = target_energy(u, t, V * 9, &en);
    if (se != GFF_OK) {
        cudaFree(x);
        cudaFree(t);
        return se;
    }
    u->sx.push_back(x);
    u->sy.push_back(t);
    u->se.push_back(en);
    u->sample_n = h->grid.nx;
    return GFF_OK;
}

// A training sample from host arrays: x [V][IN_CH], target [V][9] on an n^3 grid.
UEXPORT gff_status gff_unet_add_sample_host(gff_unet* u, int n, const float* x, const float* target) {
    if (!u || !x || !target || n < 8 || n % 8) return u ? ufail(u, GFF_ERR_ARG, "bad sample args") : GFF_ERR_ARG;
    if (u->sample_n && u->sample_n != n) return ufail(u, GFF_ERR_ARG, "all samples must share one grid");
    const long long V = (long long)n * n * n;
    std::vector<bf16> xb((size_t)V * IN_CH);
    for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16(x[i]);
    bf16* dx = nullptr;
    float* dt = nullptr;
    UTRY(cudaMalloc(&dx, xb.size() * sizeof(bf16)));
    cudaError_t e = cudaMalloc(&dt, (size_t)V * 9 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dx, xb.data(), xb.size() * sizeof(bf16), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt, target, (size_t)V * 9 * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dx);
        cudaFree(dt);
        return ufail(u, GFF_ERR_CUDA, "U-Net sample", e);
    }
    double en = 0.0;
    for (long long i = 0; i < V * 9; ++i) en += (double)target[i] * target[i];
    u->sx.push_back(dx);
    u->sy.push_back(dt);
    u->se.push_back(en / (double)(V * 9));
    u->sample_n = n;
    return GFF_OK;
}

UEXPORT int gff_unet_num_samples(const gff_unet* u) { return u ? (int)u->sx.size() : 0; }

UEXPORT gff_status gff_unet_set_sampling(gff_unet* u, int mode) {
    if (!u || mode < 0 || mode > 1) return u ? ufail(u, GFF_ERR_ARG, "sampling mode must be 0 or 1") : GFF_ERR_ARG;
    u->sampling = mode;
    return GFF_OK;
}

// Adam steps over the stored samples (one sample per step, shuffled epochs).
UEXPORT gff_status gff_unet_train(gff_unet* u, int steps, double lr, double* losses) {
    if (!u || steps < 0 || !(lr > 0)) return GFF_ERR_ARG;
    if (u->sx.empty()) return ufail(u, GFF_ERR_STATE, "no training samples");
    gff_status st = ensure_buffers(u, u->sample_n);
    if (st != GFF_OK) return st;
    const long long V = (long long)u->n * u->n * u->n;
    const int ns = (int)u->sx.size();
    std::vector<int> order(ns);
    uint64_t rs = u->seed ^ 0xA5A5A5A5ULL ^ (uint64_t)u->adam_t;
    // importance sampling: cumulative weights 1/(2 ns) + se_i / (2 sum se)
    std::vector<double> cum(ns);
    {
        double tot = 0.0;
        for (double e : u->se) tot += e;
        double c = 0.0;
        for (int i = 0; i < ns; ++i) {
            c += 0.5 / ns + (tot > 0 ? 0.5 * u->se[i] / tot : 0.5 / ns);
            cum[i] = c;
        }
    }
    for (int k = 0; k < steps; ++k) {
        int sidx;
        if (u->sampling == 1) {
            const double r = (double)(sm64(rs) >> 11) * (1.0 / 9007199254740992.0) * cum[ns - 1];
            sidx = (int)(std::upper_bound(cum.begin(), cum.end(), r) - cum.begin());
            if (sidx >= ns) sidx = ns - 1;
        } else {
            if (k % ns == 0) {  // new epoch: Fisher-Yates shuffle
                for (int i = 0; i < ns; ++i) order[i] = i;
                for (int i = ns - 1; i > 0; --i) {
                    const int j = (int)(sm64(rs) % (uint64_t)(i + 1));
                    std::swap(order[i], order[j]);
                }
            }
            sidx = order[k % ns];
        }
        View X{u->sx[sidx], IN_CH};
        if ((st = forward(u, X, nullptr)) != GFF_OK) return st;
        UTRY(cudaMemsetAsync(u->d_loss, 0, sizeof(double), nullptr));
        k_mse<<<grid_of(V * 9), 256>>>(u->Y, u->sy[sidx], u->dY, V * 9, u->d_loss);
        if ((st = backward(u, X, nullptr)) != GFF_OK) return st;
        ++u->adam_t;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)u->adam_t), c2 = 1.f - std::pow(b2, (float)u->adam_t);
        const double lr_k = lr * 0.5 * (1.0 + std::cos(M_PI * (double)k / (double)steps));  // cosine decay
        UTRY(cudaMemsetAsync(u->d_loss + 1, 0, sizeof(double), nullptr));
        k_sumsq<<<grid_of((long long)u->nparam), 256>>>(u->d_g, (long long)u->nparam, u->d_loss + 1);
        k_adam<<<grid_of((long long)u->nparam), 256>>>(u->d_w, u->d_g, u->d_m, u->d_v, (long long)u->nparam,
                                                      (float)lr_k, b1, b2, 1e-8f, c1, c2, u->d_loss + 1, GRAD_CLIP);
        if ((st = refresh_copies(u, nullptr)) != GFF_OK) return st;
        if (losses) {
            UTRY(cudaMemcpy(&losses[k], u->d_loss, sizeof(double), cudaMemcpyDeviceToHost));
        }
    }
    UTRY(cudaDeviceSynchronize());
    return GFF_OK;
}

UEXPORT gff_status gff_unet_save(gff_unet* u, const char* path) {
    if (!u || !path) return GFF_ERR_ARG;
    std::vector<float> w(gff_unet_num_params(u));
    gff_status st = gff_unet_get_params(u, w.data());
    if (st != GFF_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return ufail(u, GFF_ERR_IO, "cannot open file");
    const char magic[8] = {'G', 'F', 'F', 'U', 'N', 'E', 'T', '1'};
    const uint64_t n = w.size();
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
              std::fwrite(w.data(), sizeof(float), w.size(), f) == w.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? GFF_OK : ufail(u, GFF_ERR_IO, "write failed");
}

UEXPORT gff_status gff_unet_load(gff_unet* u, const char* path) {
    if (!u || !path) return GFF_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return ufail(u, GFF_ERR_IO, "cannot open file");
    char magic[8];
    uint64_t n = 0;
    std::vector<float> w(gff_unet_num_params(u));
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GFFUNET1", 8) == 0 && std::fread(&n, 8, 1, f) == 1 &&
              n == w.size() && std::fread(w.data(), sizeof(float), w.size(), f) == w.size();
    std::fclose(f);
    if (!ok) return ufail(u, GFF_ERR_IO, "not a U-Net weight file of this architecture");
    return gff_unet_set_params(u, w.data());
}
