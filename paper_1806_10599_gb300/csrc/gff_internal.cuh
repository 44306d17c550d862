// Internal declarations of libgff: device tables, the handle, launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "gff.h"

namespace gff {

constexpr int MAXN = 128;   // largest axis length of the plane kernels
constexpr int MAXST = 8;    // largest number of radix stages per axis
constexpr int NSLIP = 12;

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

// Mixed-radix plan of one axis: n = radix[0] * ... * radix[nst-1].
// The forward transform is decimation in frequency in place: natural input,
// output at position p holds frequency freq_of_pos(p).  The inverse replays
// the forward stages backwards with conjugate twiddles (decimation in time),
// taking that order back to natural order.
struct AxisPlan {
    int n;
    int nst;
    int radix[MAXST];
};

// Read-only tables of one grid, resident on the device.
struct GridDev {
    int nx, ny, nz, nxh;
    long long N;
    AxisPlan ax, ay, az;
    const double2* tw64[3];  // W_n^k = exp(-2 pi i k / n), k < n, per axis (x, y, z)
    const float2* tw32[3];
    const int* posx;         // [nx]: position of natural frequency kx after the forward x pass
    const int* fqy;          // [ny]: frequency held at position py after the forward y pass
    const int* fqz;          // [nz]
    const double* qt64[2][3];  // [kind][axis][k]: q~ (continuous) or q~' (discrete) per FFT index
    const float* qt32[2][3];
    long long wait_cycles;     // budget of the first wait on each bulk load (BULK_WAIT_CYCLES by default)
};

// Projection parameters of one call.
struct ProjArgs {
    int kind;        // GFF_PROJ_*
    float mask[9];   // 1 = stress-controlled component (zero frequency keeps it)
    int sym = 0;     // 1: small-strain variant, projection onto compatible symmetric fields
};

// Output epilogue of the inverse plane pass: out = scale * y + add[c].
struct OutArgs {
    double scale;
    double add[9];
};

// ---- batched launches: one launch serves several RVEs of different sizes.
// Each RVE owns the block range [start[r], start[r+1]) of the launch.
constexpr int MAX_BATCH = 64;

// One RVE's operands of a batched Galerkin apply.
struct RveApply {
    GridDev g;
    const void* x;
    const void* K;   // null: projection only
    void* y;
    void* spec;
    OutArgs oa;
    const int* skip;  // RVE stop flag, may be null
};

// One RVE's CG vectors (length n) in a batched CG launch.
struct RveVec {
    void* x;
    void* r;
    void* p;
    void* Ap;
    long long n;
};

struct GrainDev {
    const double* C;        // [ngrains][81] rotated stiffness
    const double* S0;       // [ngrains][12][9] Schmid tensors, sample frame
    const double* nrm;      // [ngrains][12][3] slip-plane normals, sample frame
    const int* kind;        // [ngrains] material kind
    const int* phase;       // [ngrains]
};

// Launch shapes of the three apply kernels (chosen by the autotuner).
struct Tune {
    int t_fwd;  // threads of k_plane_fwd
    int wz;     // (ky, kx) columns per k_zproj block
    int t_z;    // threads of k_zproj
    int t_inv;  // threads of k_plane_inv
    int inv_blocks;  // > 0: persistent streamed inverse pass with this many blocks
    int z_blocks;    // > 0: persistent TMA z pass (k_zproj_tma) with this many blocks
};

struct Nine9 {
    double v[9];
};

struct CPParamsDev {
    double gdot0, p, tau0, c, d;
    double itau0;  // 1 / tau0
    double rtol;   // return-map convergence: max_a |r_a| <= rtol
};

// Return-map tolerance for a Newton tolerance t on ||b|| / ||P||: a slip error
// dg moves P by about C dg ~ 1e3 |P| dg, so max|r| <= 1e-5 t keeps the local
// error two orders below the equilibrium tolerance; never looser than 1e-11
// nor tighter than 1e-14.
inline double return_map_tol(double newton_tol) {
    const double t = 1e-5 * newton_tol;
    return t < 1e-14 ? 1e-14 : (t > 1e-11 ? 1e-11 : t);
}

// Per-grain slip geometry block (FP64): the 12 Schmid tensors S0_a = s_a (x) m_a
// [12][9], the slip directions s_a [12][3], the 4 plane normals m_p [4][3]
// (systems 3p, 3p+1, 3p+2 share plane p) and the stiffness in Voigt order
// (11, 22, 33, 23, 13, 12) [6][6].
constexpr int GEO_S0 = 0, GEO_DIR = 108, GEO_NRM = 144, GEO_C6 = 156, GEO_STRIDE = 192;
// FP32 copies for the FP32 tangent (S0 [12][9], C [81]) and for the FP32
// pre-iteration of the return map (slip directions [12][3], plane normals
// [4][3], Voigt stiffness [6][6], the small-strain factors P [5][12] and
// C5^-1 [5][5]).
constexpr int G32_S0 = 0, G32_C = 108, G32_DIR = 189, G32_NRM = 225, G32_C6 = 237, G32_PC = 273, G32_STRIDE = 384;

}  // namespace gff

struct gff_handle {
    gff_grid grid;
    gff_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    long long N = 0;
    int nxh = 0;
    gff::GridDev g{};
    void* tables = nullptr;  // backing store of GridDev pointers

    // microstructure
    int ngrains = 0;
    bool have_ms = false;
    int* d_gid = nullptr;
    double* d_C = nullptr;
    double* d_S0 = nullptr;
    double* d_nrm = nullptr;
    float* d_geo32 = nullptr;  // [ngrains][G32_STRIDE]
    int* d_gkind = nullptr;
    int* d_gphase = nullptr;
    gff_material mat[8];
    bool mat_set[8] = {false};
    bool any_cp = false;

    // FP64 fields [9][N] (K: [81][N])
    double* d_F = nullptr;     // committed F
    double* d_Fk = nullptr;    // Newton iterate
    double* d_P = nullptr;
    double* d_K = nullptr;
    double* d_b = nullptr;
    double* d_x = nullptr;
    double* d_r = nullptr;
    double* d_p = nullptr;
    double* d_Ap = nullptr;
    // FP32 copies for the mixed path
    float* d_K32 = nullptr;
    float* d_b32 = nullptr;
    float* d_x32 = nullptr;
    float* d_r32 = nullptr;
    float* d_p32 = nullptr;
    float* d_Ap32 = nullptr;
    // half spectrum [9][nz][ny][nxh] complex (FP64 size; FP32 reuses it)
    double2* d_spec = nullptr;
    // crystal plasticity state (committed / trial) and FIP accumulators
    double* d_Fpi = nullptr;   // [9][N]
    double* d_chi = nullptr;   // [12][N]
    double* d_Fpi_t = nullptr;
    double* d_chi_t = nullptr;
    double* d_dg = nullptr;    // [12][N] slip increments of the trial
    double* d_tau = nullptr;   // [12][N]
    double* d_acc = nullptr;   // [NACC][N]
    int cp_exact_only = 0;     // 1: every return map runs the exact Newton from dg = 0 (gff_set_return_map)
    int cp_f32_first = 2;      // FP32 pre-iteration before the FP64 iteration: 1 always, 2 in mixed precision, 0 never
    int small_strain = 0;      // 1: small-strain variant: d_F holds the strain, sigma = C : eps, symmetric projection
    int* d_flag = nullptr;     // device status words: [0] CP failures, [2] timed-out bulk-copy waits,
                               // [4] return-map fallbacks, [5] local Newton iterations
    // reductions
    double* d_red = nullptr;   // partial sums
    double* d_scal = nullptr;  // final scalars
    double* h_scal = nullptr;  // pinned host mirror
    bool K_valid = false;
    bool K32_valid = false;
    bool grains_ready = false;
    void* hostdata = nullptr;  // host copies of the orientations and phases
    gff::Tune tune[2] = {{512, 8, 256, 512, 0, 0}, {512, 16, 256, 512, 0, 0}};  // [0] FP64, [1] FP32
    // tensor maps of the half spectrum for the TMA z pass: [precision][W = 8, 16], built on first use
    CUtensorMap zmap[2][2];
    bool zmap_ok[2][2] = {{false, false}, {false, false}};
    bool tuned = false;
    // warm starts: history of the completed increments.  d is an increment's
    // prescribed average F change (0 on stress-controlled components) and
    // y = (F_k - F_{k-1} - dFbar_k) / |d_k| its normalised fluctuation increment.
    float* d_gq = nullptr;       // [ngrains][5]: orientation quaternion (w, x, y, z) and phase
    float* d_yhist = nullptr;    // [2][9][N]: y of the last two completed increments
    int ycur = 0;                // slot of the last completed increment's y
    int nhist = 0;               // consecutive completed increments with |d| > 0 on record (0..2)
    double Pmacro_committed[9] = {0};  // average P of the committed state
    double cur_d9[9] = {0};      // d of the increment being solved
    double prev_d9[9] = {0};     // d of the last completed increment
    double prev2_d9[9] = {0};    // d of the one before
    struct gff_unet* unet = nullptr;
    // host-buffer apply: copy stream and its events, made on first use
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pipe_ev[18] = {};
    int pipe_nev = 0;
    std::string err;
};

namespace gff {

constexpr int NACC = 1 + 12 * 5;  // pcyc, W[12], gamma[12], gmin[12], gmax[12], sn[12]
constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs: blocks of the reductions and CG vector updates

// ---- warm starts (unet.cu): add G^(|d| y~) to h->d_Fk for the prescribed increment d9,
// y~ = s y_{k-1} (+ the network's correction when u is given).  *applied = 0 when there
// is nothing to add (|d| = 0, or extrapolation without history).
cudaError_t warm_guess(struct gff_unet* u, gff_handle* h, const double* d9, int* applied);

// ---- host helpers (api.cu)
gff_status prepare_for_increments(gff_handle* h);
// The return maps of an increment's first evaluation start from the last
// evaluated slip increments when the prescribed change d9 keeps the direction
// of the previous increment's (cosine > 1/2), else from zero.
bool first_eval_warm(const gff_handle* h, const double* d9);
// Increment history of a converged increment (h->d_Fk not yet committed):
// y = (Fk - F - dF) / |d9| into the free slot, d9 and its predecessors kept.
gff_status record_history(gff_handle* h, const double* d9, const double* dF, cudaStream_t st);
void set_error(gff_handle* h, const char* msg);

// ---- launchers (fft_proj.cu)
template <typename T>
cudaError_t launch_galerkin(const gff_handle* h, const T* x, const T* K, T* y, const ProjArgs& pa,
                            const OutArgs& oa, typename C2<T>::t* spec, cudaEvent_t* ev = nullptr,
                            const int* skip = nullptr);
// the apply from host x_host to host y_host through the device buffers xd, yd,
// pipelined over chunks of z-planes (copy stream + events of the handle)
template <typename T>
cudaError_t launch_galerkin_host(gff_handle* h, const T* x_host, T* y_host, T* xd, T* yd, const T* K,
                                 const ProjArgs& pa, const OutArgs& oa, typename C2<T>::t* spec);
size_t plane_smem_bytes(int nx, int ny, int elem);
// Mixed-radix plan of one axis (false: n unsupported) and the frequency held
// at position pos after the forward (decimation in frequency) transform:
// pos = sum_i p_i m_i with m_i = n / (r_0 ... r_i), frequency p_0 + r_0 p_1 + ...
bool make_axis_plan(int n, AxisPlan& p);
int axis_freq_of_pos(int pos, const AxisPlan& p);
// Blocks of the z pass: one per tensor row (3) and W (ky, kx) columns.
inline int zproj_blocks(const GridDev& g, int W) { return 3 * (int)(((long long)g.ny * g.nxh + W - 1) / W); }
// Times every candidate launch shape of the three kernels on the handle's own
// buffers and stores the fastest in h->tune (results do not depend on it).
cudaError_t autotune_galerkin(gff_handle* h);
// Launch shapes chosen by the caller; false (nothing changed) if a shape is unsupported.
bool set_tiles(gff_handle* h, const Tune& t64, const Tune& t32);

// Batched apply: rv (device, n entries), start arrays (device) for the plane
// kernels (9 nz blocks per RVE) and the z kernel (zproj_blocks per RVE).
struct BatchLaunch {
    int n;
    const RveApply* rv;
    const int* start_plane;
    const int* start_z;
    int blocks_plane, blocks_z;
    size_t smem_plane, smem_z;
    Tune tn;
    bool vin, vout, withK;
};
template <typename T>
cudaError_t launch_galerkin_batch(const BatchLaunch& bl, const ProjArgs& pa, cudaStream_t st);
template <typename T> size_t batch_z_smem(const GridDev& g, int W);

// ---- vector kernels (vec.cu)
template <typename T>
cudaError_t launch_dot(const T* a, const T* b, long long n, double* partial, double* out, cudaStream_t s);
cudaError_t launch_sum9(const double* a, long long N, double* partial, double* out9, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_update(T* x, T* r, const T* p, const T* Ap, double alpha, long long n, double* partial,
                             double* out_rr, cudaStream_t s);
template <typename T>
cudaError_t launch_xpby(T* p, const T* r, double beta, long long n, cudaStream_t s);
cudaError_t launch_add_const9(double* F, const double* Fsrc, const double* d9, long long N, cudaStream_t s);
template <typename Tin>
cudaError_t launch_axpy_to64(double* y, const Tin* x, long long n, cudaStream_t s);
cudaError_t launch_cast64to32(float* y, const double* x, long long n, cudaStream_t s);
// y[c][v] = (Fk[c][v] - F[c][v] - dF9[c]) * inv   (normalised fluctuation increment, FP32)
cudaError_t launch_fluct_incr(float* y, const double* Fk, const double* F, const double* dF9, double inv, long long N,
                              cudaStream_t s);
cudaError_t launch_fill(double* y, double v, long long n, cudaStream_t s);
// Device-resident CG scalars (see vec.cu): cg[CG_RR] = r.r, cg[CG_PAP], cg[CG_ALPHA],
// cg[CG_BETA], cg[CG_STOP2] = stop^2, cg[CG_ITERS]; flag[0] = stop, flag[1] = breakdown.
enum { CG_RR = 0, CG_PAP = 1, CG_ALPHA = 2, CG_BETA = 3, CG_STOP2 = 4, CG_ITERS = 5 };
// flag[CG_TICKET_*]: the last-block tickets of the two CG reductions (0 between launches)
enum { CG_TICKET_ALPHA = 4, CG_TICKET_BETA = 5 };
cudaError_t launch_cg_init(double* cg, int* flag, double rr0, double stop2, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_alpha(const T* p, const T* Ap, long long n, double* partial, double* cg, int* flag,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_cg_step(T* x, T* r, T* p, const T* Ap, long long n, double* partial, double* cg, int* flag,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_zero(T* y, long long n, cudaStream_t s);

// measurement helpers (vec.cu): FP64 FMA throughput; durations of the CG vector kernels
cudaError_t measure_fp64_fma(double* out, int blocks, int iters, int reps, cudaStream_t s, double* gflops,
                             float* ms_best);
template <typename T>
cudaError_t time_cg_kernels(T* x, T* r, T* p, T* Ap, long long n, double* partial, double* cg, int* flag,
                            cudaStream_t s, int reps, float* ms);

// batched CG (per-RVE scalars cg[r * 8 + CG_*], flags[2 r], flags[2 r + 1])
cudaError_t launch_cg_init_batch(int n, double* cg, int* flag, const double* rr0_stop2_dev, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_alpha_batch(int n, const RveVec* v, double* partial, double* cg, int* flag, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_step_batch(int n, const RveVec* v, double* partial, double* cg, int* flag, cudaStream_t s);
// out[r] = a_r . b_r for the n pairs (a_r, b_r) = (v[r].x, v[r].r); partial holds n * RED_BLOCKS
template <typename T>
cudaError_t launch_dot_batch(int n, const RveVec* v, double* partial, double* out, cudaStream_t s);
size_t batch_plane_smem(int nx, int ny, int elem);

// ---- constitutive kernels (material.cu)
// tangent: TANGENT_F64 writes the FP64 K; TANGENT_F64_AND_F32 also rounds it into K32;
// TANGENT_F32 computes the crystal-plasticity tangent in FP32 and writes only K32.
// warm: start each voxel's local Newton from the slip increments left in d_dg by the previous call.
enum { TANGENT_F64 = 0, TANGENT_F64_AND_F32 = 1, TANGENT_F32 = 2 };
// part: CONST_ALL (P and K), CONST_P (return map and P; K untouched), CONST_K (K at
// the slips the last CONST_P launch stored; P and the trial state untouched).
enum { CONST_ALL = 0, CONST_P = 1, CONST_K = 2 };
cudaError_t launch_constitutive(gff_handle* h, const double* F, double dt, int tangent, bool warm = false,
                                int part = CONST_ALL);
cudaError_t launch_fip_accumulate(gff_handle* h);
cudaError_t preload_constitutive();
// Batched constitutive update of the RVEs hs[0..n): the per-RVE arguments are
// uploaded once (skip_dev[2 r] != 0: RVE r is left alone; cpflag_dev[r] counts
// its return-map failures; warm[r] or, when warm_dev is set, warm_dev[r] != 0
// at run time starts its return maps from the stored slips), then launched as
// often as needed -- also inside a captured graph.
cudaError_t upload_constitutive_batch(gff_handle* const* hs, int n, double dt, int tangent, const bool* warm,
                                      const int* warm_dev, const int* skip_dev, int* cpflag_dev, void* scratch_dev,
                                      int* blocks_out, cudaStream_t st);
cudaError_t launch_constitutive_batch_uploaded(const void* scratch_dev, int n, int blocks, int tangent, int part,
                                               cudaStream_t st);
size_t constitutive_batch_scratch_bytes();
cudaError_t launch_fip_reset(gff_handle* h);
// Appendix A: (F, Cauchy stress, Jaumann-rate tangent C^ab) -> (P, K) for n voxels, SoA [9][n] / [81][n]
cudaError_t launch_umat_convert(long long n, const double* F, const double* sigma, const double* Cab, double* P,
                                double* K, cudaStream_t st);
// band-averaged W_cyc (Eq. Wmax) per grain into out[ngrains] (device), NB bands per plane
size_t band_scratch_bytes(int ngrains, int NB);
cudaError_t launch_band_fips(gff_handle* h, double width, int NB, void* scratch, double* out);
cudaError_t launch_grain_fips(gff_handle* h, double* pc, double* w, double* fs);

}  // namespace gff
