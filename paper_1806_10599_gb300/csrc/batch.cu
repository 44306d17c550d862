// Batched increments of several RVEs of different sizes (gff_batch_run).
//
// All RVEs follow one macroscopic loading history.  Each load increment is
// ONE launch of a CUDA graph whose Newton-Raphson and conjugate-gradient loops
// (Sect. 2.1) run on the device as conditional WHILE nodes:
//
//   WHILE any RVE is still iterating (at most newton_max + 1 times):
//     constitutive update P of the iterating RVEs          (one launch, all RVEs)
//     residual b = -G_M(P) + M : Pbar                      (per size class)
//     norms ||b||, ||P||; Newton decision per RVE         (converged / failed / correct)
//     tangent K of the RVEs taking a correction            (one launch)
//     right-hand side, CG start
//     WHILE any CG is running (at most cg_max times):
//       apply G_M(K : p)                                   (per size class)
//       CG vector updates                                  (one launch each)
//     F += dF for the RVEs whose CG did not break down
//
// Per-RVE status words, Newton and CG counters live on the device, so RVEs
// converge independently and a finished RVE's blocks return at entry; the
// host reads them once per increment.  RVEs are grouped by grid size: each
// size class runs the three apply kernels with the launch shapes the
// autotuner chose for it, on a stream of its own inside the graph, so the
// classes overlap.  An RVE whose increment fails in the batch (return map,
// Newton or CG) is redone by gff_step on its own handle -- with its cut-backs
// -- before the next increment.  The extrapolated warm start (mode 3) is
// applied per RVE before the graph runs.  Each RVE's arithmetic (including
// every reduction's block structure) is exactly that of gff_step on its own
// handle, so an RVE that converges in the batch gets the one-by-one result
// bit for bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "gff_internal.cuh"

using namespace gff;

namespace {

enum { ST_ACTIVE = 0, ST_DONE = 1, ST_FAILED = 2, ST_IDLE = 3 };

// Right-hand side and update pointers of one RVE (vectors in the solve precision).
struct RveRhs {
    const double* b;  // residual (FP64)
    void* r;
    void* x;
    void* p;
    double* Fk;  // Newton iterate
    long long n;  // 9 N
};

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// RVEs with the same grid: one set of batched apply launches with their own
// shapes, on streams of their own ([0] residual, [1] CG apply).
struct SizeClass {
    std::vector<int> rves;
    BatchLaunch res{}, cg{};
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
};

// int words of the per-increment state block: status, skip flags, counters
struct StateLayout {
    int stat, inactive, ksk, cpflag, kflag, newton, cgsum, warm, ctr, total;
    explicit StateLayout(int n) {
        int o = 0;
        stat = o, o += n;
        inactive = o, o += 2 * n;  // stride 2, like the CG flags
        ksk = o, o += 2 * n;       // 0: the RVE takes a Newton correction this iteration
        cpflag = o, o += n;        // return-map failures of the evaluation (then kflag: of the tangent)
        kflag = o, o += n;
        newton = o, o += n;
        cgsum = o, o += n;
        warm = o, o += n;          // 1 after the first evaluation: return maps start warm
        ctr = o, o += 4;           // [0] Newton bodies run, [1] CG iterations run
        total = o;
    }
};

struct Batch {
    int n = 0;
    cudaStream_t st = nullptr;
    cudaStream_t cap[2] = {nullptr, nullptr};  // capture streams of the two loop bodies
    cudaStream_t saved[MAX_BATCH];
    gff_handle* h[MAX_BATCH];
    bool mixed = false;
    DevBuf arena;
    RveApply* d_res = nullptr;   // [n] residual-apply descriptors, grouped by class
    RveApply* d_cga = nullptr;   // [n] CG-apply descriptors, grouped by class
    int* d_starts = nullptr;     // per class: plane and z block prefixes
    RveVec* d_vec = nullptr;     // CG vectors in the solve precision
    RveVec* d_nb = nullptr;      // (b, b)
    RveVec* d_nP = nullptr;      // (P, P)
    RveVec* d_nr32 = nullptr;    // (r32, r32)
    RveRhs* d_rhs = nullptr;
    double* d_cg = nullptr;      // [n][8] CG scalars
    int* d_cgflag = nullptr;     // [n][2] CG stop / breakdown
    int* d_state = nullptr;      // per-increment state block (StateLayout)
    double* d_partial = nullptr; // [max(n, 9)][RED_BLOCKS]
    double* d_out = nullptr;     // [18 n]
    double* d_dvals = nullptr;   // [4 n]: residual, first residual, stop^2
    void* d_cargsP = nullptr;    // uploaded constitutive arguments (return map and P)
    void* d_cargsK = nullptr;    // (tangent)
    int blocksP = 0, blocksK = 0;
    double* h_pin = nullptr;
    std::vector<SizeClass> cls;
    cudaEvent_t fork[2] = {nullptr, nullptr};
    std::map<unsigned, cudaGraphExec_t> graphs;  // by stress-control mask
    std::vector<cudaGraph_t> graph_defs;

    ~Batch() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        for (cudaGraph_t gr : graph_defs) cudaGraphDestroy(gr);
        for (auto& c : cls)
            for (int i = 0; i < 2; ++i) {
                if (c.done[i]) cudaEventDestroy(c.done[i]);
                if (c.s[i]) cudaStreamDestroy(c.s[i]);
            }
        for (cudaEvent_t f : fork)
            if (f) cudaEventDestroy(f);
        if (h_pin) cudaFreeHost(h_pin);
        for (int r = 0; r < n; ++r) h[r]->stream = saved[r];
        for (cudaStream_t c : cap)
            if (c) cudaStreamDestroy(c);
        if (st) cudaStreamDestroy(st);
    }
};

gff_status cuda_fail(gff_handle* h, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "batch %s: %s", what, cudaGetErrorString(e));
    set_error(h, buf);
    return GFF_ERR_CUDA;
}

#define BTRY(expr)                                                  \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return cuda_fail(B.h[0], e_, #expr); \
    } while (0)

template <typename T> bool vec_aligned(const GridDev& g, const void* p) {
    return (g.nx % (16 / (int)sizeof(T))) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// ---------------------------------------------------------------- device-side Newton / CG control
constexpr int CTL_THREADS = MAX_BATCH;  // one thread per RVE

// Newton decision after the residual norms (what gff_step decides on the host):
// converged, failed (return map, non-finite residual, iteration cap) or a
// correction by CG stopping at max(cg_tol ||b||, 0.1 newton_tol ||P||).
__global__ void __launch_bounds__(CTL_THREADS) k_decide(int n, const double* __restrict__ out, int* st, StateLayout L,
                                                       double* __restrict__ dv, double newton_tol, double cg_tol,
                                                       int newton_max) {
    const int r = threadIdx.x;
    if (r >= n) return;
    int* stat = st + L.stat;
    int* ksk = st + L.ksk;
    int* ina = st + L.inactive;
    ksk[2 * r] = 1;
    if (stat[r] != ST_ACTIVE) return;
    const bool first = st[L.warm + r] == 0;
    st[L.warm + r] = 1;  // later return maps start from the slips of this evaluation
    if (st[L.cpflag + r]) {
        stat[r] = ST_FAILED;
        ina[2 * r] = 1;
        return;
    }
    const double nb = sqrt(out[r]), nP = sqrt(out[n + r]);
    const double res = nP > 0 ? nb / nP : nb;
    dv[r] = res;
    if (first) dv[n + r] = res;
    if (res <= newton_tol) {
        stat[r] = ST_DONE;
        ina[2 * r] = 1;
        return;
    }
    if (!isfinite(res) || st[L.newton + r] == newton_max) {
        stat[r] = ST_FAILED;
        ina[2 * r] = 1;
        return;
    }
    const double stop = fmax(cg_tol * nb, 0.1 * newton_tol * nP);
    dv[2 * n + r] = stop * stop;
    ksk[2 * r] = 0;
}

// a tangent that failed ends the RVE's increment in the batch
__global__ void __launch_bounds__(CTL_THREADS) k_tangent_check(int n, int* st, StateLayout L) {
    const int r = threadIdx.x;
    if (r >= n || st[L.ksk + 2 * r] || !st[L.kflag + r]) return;
    st[L.stat + r] = ST_FAILED;
    st[L.inactive + 2 * r] = 1;
    st[L.ksk + 2 * r] = 1;
}

// r = b (rounded to T), x = 0, p = r for the RVEs taking a correction; grid (blocks, n)
template <typename T>
__global__ void __launch_bounds__(256) k_rhs(const RveRhs* __restrict__ rh, const int* __restrict__ st, StateLayout L) {
    const int r = blockIdx.y;
    if (st[L.ksk + 2 * r]) return;
    const RveRhs a = rh[r];
    T* rr = static_cast<T*>(a.r);
    T* x = static_cast<T*>(a.x);
    T* p = static_cast<T*>(a.p);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        const T v = (T)a.b[i];
        rr[i] = v;
        x[i] = (T)0;
        p[i] = v;
    }
}

// CG scalars and stop flags of every RVE (r.r = rr0, stop on r.r <= stop^2); the
// CG loop is entered when some RVE's solve has to run
__global__ void __launch_bounds__(CTL_THREADS) k_cg_start(int n, const double* __restrict__ rr0,
                                                         const double* __restrict__ dv, int* st, StateLayout L,
                                                         double* cg, int* flag, cudaGraphConditionalHandle hc) {
    const int r = threadIdx.x;
    bool go = false;
    if (r < n) {
        const bool solving = st[L.ksk + 2 * r] == 0;
        const double a = rr0[r], s2 = dv[2 * n + r];
        double* c = cg + 8 * r;
        c[CG_RR] = a;
        c[CG_PAP] = 0.0;
        c[CG_ALPHA] = 0.0;
        c[CG_BETA] = 0.0;
        c[CG_STOP2] = s2;
        c[CG_ITERS] = 0.0;
        flag[2 * r] = (!solving || a <= s2) ? 1 : 0;
        flag[2 * r + 1] = 0;
        go = flag[2 * r] == 0;
    }
    go = __syncthreads_or(go);
    if (threadIdx.x == 0) {
        st[L.ctr + 1] = 0;
        cudaGraphSetConditional(hc, go ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(CTL_THREADS) k_cg_more(int n, const int* __restrict__ flag, int* st, StateLayout L,
                                                        int cg_max, cudaGraphConditionalHandle hc) {
    const int r = threadIdx.x;
    const bool go = __syncthreads_or(r < n && flag[2 * r] == 0);
    if (threadIdx.x == 0) {
        const int it = ++st[L.ctr + 1];
        cudaGraphSetConditional(hc, (go && it < cg_max) ? 1u : 0u);
    }
}

// F += dF for the RVEs whose CG did not break down; grid (blocks, n)
template <typename T>
__global__ void __launch_bounds__(256) k_newton_update(const RveRhs* __restrict__ rh, const int* __restrict__ st,
                                                      StateLayout L, const int* __restrict__ flag) {
    const int r = blockIdx.y;
    if (st[L.ksk + 2 * r] || flag[2 * r + 1]) return;
    const RveRhs a = rh[r];
    const T* x = static_cast<const T*>(a.x);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x)
        a.Fk[i] += (double)x[i];
}

// counters of the corrected RVEs; the Newton loop goes on while any RVE iterates
__global__ void __launch_bounds__(CTL_THREADS) k_newton_more(int n, int* st, StateLayout L, const int* __restrict__ flag,
                                                            const double* __restrict__ cg, int newton_max,
                                                            cudaGraphConditionalHandle hn) {
    const int r = threadIdx.x;
    if (r < n && st[L.ksk + 2 * r] == 0) {
        if (flag[2 * r + 1]) {
            st[L.stat + r] = ST_FAILED;
            st[L.inactive + 2 * r] = 1;
        } else {
            st[L.newton + r] += 1;
            st[L.cgsum + r] += (int)cg[8 * r + CG_ITERS];
        }
    }
    const bool go = __syncthreads_or(r < n && st[L.stat + r] == ST_ACTIVE);
    if (threadIdx.x == 0) {
        const int it = ++st[L.ctr];
        cudaGraphSetConditional(hn, (go && it < newton_max + 1) ? 1u : 0u);
    }
}

inline int vec_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 152LL * 4 ? (b < 1 ? 1 : b) : 152LL * 4);
}

// ---------------------------------------------------------------- set-up
// Launch description of the batched apply of one size class over d_rv[0..m).
template <typename T>
BatchLaunch class_launch(const std::vector<RveApply>& rv, RveApply* d_rv, int* d_start_pl, int* d_start_z,
                         const Tune& tn, bool withK, std::vector<int>& start_pl, std::vector<int>& start_z) {
    const int m = (int)rv.size();
    BatchLaunch bl{};
    bl.n = m;
    bl.rv = d_rv;
    bl.tn = tn;
    // the batched passes run the one-block-per-strip z kernel (at most 256 threads) and
    // the one-block-per-plane inverse (at most 512): persistent shapes map onto them,
    // and every shape gives the same bits
    bl.tn.t_fwd = std::abs(bl.tn.t_fwd);  // (negative: the register-staged pass of one handle)
    bl.tn.t_z = std::min(bl.tn.t_z, 256);
    bl.tn.t_inv = std::min(bl.tn.t_inv, 512);
    bl.withK = withK;
    bl.vin = bl.vout = true;
    start_pl.assign(m + 1, 0);
    start_z.assign(m + 1, 0);
    for (int r = 0; r < m; ++r) {
        const GridDev& g = rv[r].g;
        start_pl[r + 1] = start_pl[r] + 9 * g.nz;
        start_z[r + 1] = start_z[r] + zproj_blocks(g, bl.tn.wz);
        bl.smem_plane = std::max(bl.smem_plane, batch_plane_smem(g.nx, g.ny, (int)sizeof(typename C2<T>::t)));
        bl.smem_z = std::max(bl.smem_z, batch_z_smem<T>(g, bl.tn.wz));
        bl.vin = bl.vin && vec_aligned<T>(g, rv[r].x) && (!withK || vec_aligned<T>(g, rv[r].K));
        bl.vout = bl.vout && vec_aligned<T>(g, rv[r].y);
    }
    bl.start_plane = d_start_pl;
    bl.start_z = d_start_z;
    bl.blocks_plane = start_pl[m];
    bl.blocks_z = start_z[m];
    return bl;
}

gff_status setup(Batch& B) {
    const int n = B.n;
    const gff_options& o = B.h[0]->opt;
    B.mixed = o.precision == GFF_PREC_MIXED;
    // size classes (RVEs with the same grid), in order of first appearance
    for (int r = 0; r < n; ++r) {
        const gff_grid& gr = B.h[r]->grid;
        int c = 0;
        for (; c < (int)B.cls.size(); ++c) {
            const gff_grid& g0 = B.h[B.cls[c].rves[0]]->grid;
            if (g0.nx == gr.nx && g0.ny == gr.ny && g0.nz == gr.nz) break;
        }
        if (c == (int)B.cls.size()) B.cls.emplace_back();
        B.cls[c].rves.push_back(r);
    }
    const int ncls = (int)B.cls.size();
    const StateLayout L(n);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t a = off;
        off += (bytes + 255) / 256 * 256;
        return a;
    };
    const size_t o_res = take(sizeof(RveApply) * n), o_cga = take(sizeof(RveApply) * n);
    const size_t o_st = take(sizeof(int) * 3 * (n + ncls));
    const size_t o_vec = take(sizeof(RveVec) * n), o_nb = take(sizeof(RveVec) * n), o_nP = take(sizeof(RveVec) * n);
    const size_t o_nr32 = take(sizeof(RveVec) * n), o_rhs = take(sizeof(RveRhs) * n);
    const size_t o_cg = take(sizeof(double) * 8 * n), o_cgf = take(sizeof(int) * 2 * n);
    const size_t o_state = take(sizeof(int) * L.total);
    const size_t o_part = take(sizeof(double) * RED_BLOCKS * std::max(n, 9));
    const size_t o_out = take(sizeof(double) * 18 * n), o_dv = take(sizeof(double) * 4 * n);
    const size_t o_cp = take(constitutive_batch_scratch_bytes()), o_ck = take(constitutive_batch_scratch_bytes());
    BTRY(cudaMalloc(&B.arena.p, off));
    unsigned char* d = static_cast<unsigned char*>(B.arena.p);
    B.d_res = reinterpret_cast<RveApply*>(d + o_res);
    B.d_cga = reinterpret_cast<RveApply*>(d + o_cga);
    B.d_starts = reinterpret_cast<int*>(d + o_st);
    B.d_vec = reinterpret_cast<RveVec*>(d + o_vec);
    B.d_nb = reinterpret_cast<RveVec*>(d + o_nb);
    B.d_nP = reinterpret_cast<RveVec*>(d + o_nP);
    B.d_nr32 = reinterpret_cast<RveVec*>(d + o_nr32);
    B.d_rhs = reinterpret_cast<RveRhs*>(d + o_rhs);
    B.d_cg = reinterpret_cast<double*>(d + o_cg);
    B.d_cgflag = reinterpret_cast<int*>(d + o_cgf);
    B.d_state = reinterpret_cast<int*>(d + o_state);
    B.d_partial = reinterpret_cast<double*>(d + o_part);
    B.d_out = reinterpret_cast<double*>(d + o_out);
    B.d_dvals = reinterpret_cast<double*>(d + o_dv);
    B.d_cargsP = d + o_cp;
    B.d_cargsK = d + o_ck;
    BTRY(cudaMallocHost(&B.h_pin, sizeof(double) * (64 * std::max(n, 4)) + sizeof(int) * L.total));

    std::vector<RveApply> res(n), cga(n);
    std::vector<RveVec> vec(n), nb(n), nP(n), nr32(n);
    std::vector<RveRhs> rhs(n);
    for (int r = 0; r < n; ++r) {
        gff_handle* h = B.h[r];
        const long long n9 = 9 * h->N;
        if (B.mixed) {
            vec[r] = {h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, n9};
            rhs[r] = {h->d_b, h->d_r32, h->d_x32, h->d_p32, h->d_Fk, n9};
        } else {
            vec[r] = {h->d_x, h->d_r, h->d_p, h->d_Ap, n9};
            rhs[r] = {h->d_b, h->d_r, h->d_x, h->d_p, h->d_Fk, n9};
        }
        nb[r] = {h->d_b, h->d_b, nullptr, nullptr, n9};
        nP[r] = {h->d_P, h->d_P, nullptr, nullptr, n9};
        nr32[r] = {h->d_r32, h->d_r32, nullptr, nullptr, n9};
    }
    // descriptors grouped by class: class c owns [cbase, cbase + |c|) of d_res / d_cga
    std::vector<int> starts;
    int cbase = 0;
    for (int c = 0; c < ncls; ++c) {
        SizeClass& sc = B.cls[c];
        const int m = (int)sc.rves.size();
        std::vector<RveApply> rc, gc;
        for (int r : sc.rves) {
            gff_handle* h = B.h[r];
            RveApply a{};
            a.g = h->g;
            a.x = h->d_P;
            a.K = nullptr;
            a.y = h->d_b;
            a.spec = h->d_spec;
            a.skip = B.d_state + L.inactive + 2 * r;
            rc.push_back(a);
            RveApply q{};
            q.g = h->g;
            q.spec = h->d_spec;
            q.oa.scale = 1.0 / (double)h->N;
            for (int k = 0; k < 9; ++k) q.oa.add[k] = 0.0;
            q.skip = B.d_cgflag + 2 * r;
            q.x = B.mixed ? (void*)h->d_p32 : (void*)h->d_p;
            q.K = B.mixed ? (void*)h->d_K32 : (void*)h->d_K;
            q.y = B.mixed ? (void*)h->d_Ap32 : (void*)h->d_Ap;
            gc.push_back(q);
        }
        int* spl = B.d_starts + (int)starts.size();
        int* szr = spl + (m + 1);
        int* szc = szr + (m + 1);
        std::vector<int> s_pl, s_zr, s_zc;
        const gff_handle* rep = B.h[sc.rves[0]];  // the class's own tuned shapes
        sc.res = class_launch<double>(rc, B.d_res + cbase, spl, szr, rep->tune[0], false, s_pl, s_zr);
        if (B.mixed)
            sc.cg = class_launch<float>(gc, B.d_cga + cbase, spl, szc, rep->tune[1], true, s_pl, s_zc);
        else
            sc.cg = class_launch<double>(gc, B.d_cga + cbase, spl, szc, rep->tune[0], true, s_pl, s_zc);
        starts.insert(starts.end(), s_pl.begin(), s_pl.end());
        starts.insert(starts.end(), s_zr.begin(), s_zr.end());
        starts.insert(starts.end(), s_zc.begin(), s_zc.end());
        for (int i = 0; i < m; ++i) {
            res[cbase + i] = rc[i];
            cga[cbase + i] = gc[i];
        }
        cbase += m;
        for (int i = 0; i < 2; ++i) {
            BTRY(cudaStreamCreateWithFlags(&sc.s[i], cudaStreamNonBlocking));
            BTRY(cudaEventCreateWithFlags(&sc.done[i], cudaEventDisableTiming));
        }
    }
    for (int i = 0; i < 2; ++i) {
        BTRY(cudaEventCreateWithFlags(&B.fork[i], cudaEventDisableTiming));
        BTRY(cudaStreamCreateWithFlags(&B.cap[i], cudaStreamNonBlocking));
    }
    BTRY(cudaMemcpyAsync(B.d_res, res.data(), sizeof(RveApply) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_cga, cga.data(), sizeof(RveApply) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_starts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_vec, vec.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nb, nb.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nP, nP.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nr32, nr32.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_rhs, rhs.data(), sizeof(RveRhs) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaStreamSynchronize(B.st));  // the host vectors above go out of scope
    return GFF_OK;
}

// Output epilogue of the residual projection b = -G_M(P) + M : Pbar: -1/N and
// the mask term; set once per increment (Pbar and the mask may change).
gff_status set_residual_epilogue(Batch& B, const double* add9) {
    std::vector<OutArgs> oa(B.n);
    int pos = 0;
    for (const SizeClass& sc : B.cls)
        for (int r : sc.rves) {
            OutArgs& o = oa[pos++];
            o.scale = -1.0 / (double)B.h[r]->N;
            for (int c = 0; c < 9; ++c) o.add[c] = add9[c];
        }
    for (int i = 0; i < B.n; ++i)
        BTRY(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(B.d_res + i) + offsetof(RveApply, oa), &oa[i],
                             sizeof(OutArgs), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaStreamSynchronize(B.st));
    return GFF_OK;
}

// ---------------------------------------------------------------- the increment graph
// The apply of every size class on its own stream, forked from and joined to s.
template <typename T>
cudaError_t apply_classes(Batch& B, int which, const ProjArgs& pa, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(B.fork[which], s);
    for (SizeClass& sc : B.cls) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sc.s[which], B.fork[which], 0);
        if (e == cudaSuccess) e = launch_galerkin_batch<T>(which ? sc.cg : sc.res, pa, sc.s[which]);
        if (e == cudaSuccess) e = cudaEventRecord(sc.done[which], sc.s[which]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, sc.done[which], 0);
    }
    return e;
}

// The graph being captured on s.
cudaError_t capture_graph(cudaStream_t s, cudaGraph_t* g) {
    cudaStreamCaptureStatus cs;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr);
    if (e == cudaSuccess && cs != cudaStreamCaptureStatusActive) e = cudaErrorIllegalState;
    return e;
}

// Appends a WHILE node on `handle` to the capture on s; returns its body graph.
cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle handle, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorIllegalState;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = handle;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &p)) != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

template <typename T>
cudaError_t capture_cg_body(Batch& B, const ProjArgs& pa, cudaStream_t s, cudaGraphConditionalHandle hc) {
    const StateLayout L(B.n);
    cudaError_t e = apply_classes<T>(B, 1, pa, s);
    if (e == cudaSuccess) e = launch_cg_alpha_batch<T>(B.n, B.d_vec, B.d_partial, B.d_cg, B.d_cgflag, s);
    if (e == cudaSuccess) e = launch_cg_step_batch<T>(B.n, B.d_vec, B.d_partial, B.d_cg, B.d_cgflag, s);
    if (e != cudaSuccess) return e;
    k_cg_more<<<1, CTL_THREADS, 0, s>>>(B.n, B.d_cgflag, B.d_state, L, B.h[0]->opt.cg_max, hc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t capture_newton_body(Batch& B, const ProjArgs& pa, cudaStream_t s, cudaGraphConditionalHandle hn) {
    const int n = B.n;
    const StateLayout L(n);
    const gff_options& o = B.h[0]->opt;
    const int tangent = B.mixed ? TANGENT_F32 : TANGENT_F64;
    int* st = B.d_state;
    cudaError_t e = cudaMemsetAsync(st + L.cpflag, 0, 2 * n * sizeof(int), s);  // cpflag and kflag
    if (e == cudaSuccess) e = launch_constitutive_batch_uploaded(B.d_cargsP, n, B.blocksP, tangent, CONST_P, s);
    if (e == cudaSuccess) e = apply_classes<double>(B, 0, pa, s);
    if (e == cudaSuccess) e = launch_dot_batch<double>(n, B.d_nb, B.d_partial, B.d_out, s);
    if (e == cudaSuccess) e = launch_dot_batch<double>(n, B.d_nP, B.d_partial, B.d_out + n, s);
    if (e != cudaSuccess) return e;
    k_decide<<<1, CTL_THREADS, 0, s>>>(n, B.d_out, st, L, B.d_dvals, o.newton_tol, o.cg_tol, o.newton_max);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_constitutive_batch_uploaded(B.d_cargsK, n, B.blocksK, tangent, CONST_K, s)) != cudaSuccess) return e;
    k_tangent_check<<<1, CTL_THREADS, 0, s>>>(n, st, L);
    long long nmax = 0;
    for (int r = 0; r < n; ++r) nmax = std::max(nmax, 9 * B.h[r]->N);
    k_rhs<T><<<dim3(vec_blocks(nmax), n), 256, 0, s>>>(B.d_rhs, st, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double* rr0 = B.d_out;  // FP64: r.r = b.b of the decision
    if (B.mixed) {                // the FP32 solve starts from the rounded residual
        if ((e = launch_dot_batch<float>(n, B.d_nr32, B.d_partial, B.d_out + 2 * n, s)) != cudaSuccess) return e;
        rr0 = B.d_out + 2 * n;
    }
    cudaGraph_t outer, body;
    cudaGraphConditionalHandle hc;
    if ((e = capture_graph(s, &outer)) != cudaSuccess) return e;
    if ((e = cudaGraphConditionalHandleCreate(&hc, outer, 0, 0)) != cudaSuccess) return e;
    k_cg_start<<<1, CTL_THREADS, 0, s>>>(n, rr0, B.d_dvals, st, L, B.d_cg, B.d_cgflag, hc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = add_while(s, hc, &body)) != cudaSuccess) return e;
    cudaStream_t sc = B.cap[1];
    if ((e = cudaStreamBeginCaptureToGraph(sc, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
    e = capture_cg_body<T>(B, pa, sc, hc);
    cudaGraph_t got = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(sc, &got);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    k_newton_update<T><<<dim3(vec_blocks(nmax), n), 256, 0, s>>>(B.d_rhs, st, L, B.d_cgflag);
    k_newton_more<<<1, CTL_THREADS, 0, s>>>(n, st, L, B.d_cgflag, B.d_cg, o.newton_max, hn);
    return cudaGetLastError();
}

// The executable graph of one increment for a stress-control mask (built once per mask).
gff_status increment_graph(Batch& B, const ProjArgs& pa, unsigned key, cudaGraphExec_t* out) {
    auto it = B.graphs.find(key);
    if (it != B.graphs.end()) {
        *out = it->second;
        return GFF_OK;
    }
    cudaStream_t s = B.st;
    BTRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    cudaGraph_t top = nullptr, body = nullptr;
    cudaGraphConditionalHandle hn;
    cudaError_t e = capture_graph(s, &top);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hn, top, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = add_while(s, hn, &body);
    if (e == cudaSuccess) {
        cudaStream_t sn = B.cap[0];
        e = cudaStreamBeginCaptureToGraph(sn, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            e = B.mixed ? capture_newton_body<float>(B, pa, sn, hn) : capture_newton_body<double>(B, pa, sn, hn);
            cudaGraph_t got = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(sn, &got);
            if (e == cudaSuccess) e = e2;
        }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e3 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e3;
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(B.h[0], e, "increment graph capture");
    }
    B.graph_defs.push_back(g);
    B.graphs[key] = ex;
    *out = ex;
    return GFF_OK;
}

// ---------------------------------------------------------------- increments
// Commit of a converged RVE, as gff_step commits: increment history (mean F
// change from the sums of the iterate and of the committed F), state, FIPs.
gff_status commit_rve(Batch& B, int r, const double* Fsum) {
    gff_handle* h = B.h[r];
    const long long N = h->N;
    double dF[9];
    BTRY(launch_sum9(h->d_Fk, N, B.d_partial, B.d_out, B.st));
    BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, B.st));
    BTRY(cudaStreamSynchronize(B.st));
    for (int c = 0; c < 9; ++c) dF[c] = (B.h_pin[c] - Fsum[c]) / (double)N;
    gff_status sh = record_history(h, h->cur_d9, dF, B.st);
    if (sh != GFF_OK) return sh;
    BTRY(cudaMemcpyAsync(h->d_F, h->d_Fk, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
    if (h->any_cp) {
        BTRY(cudaMemcpyAsync(h->d_Fpi, h->d_Fpi_t, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
        BTRY(cudaMemcpyAsync(h->d_chi, h->d_chi_t, 12 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
        BTRY(launch_fip_accumulate(h));
    }
    h->K_valid = h->K32_valid = false;  // the converged iterate's tangent is not computed
    return GFF_OK;
}

gff_status run(Batch& B, int nsteps, const double* dt, const double* Fbar, const uint8_t* mask, const double* Pbar,
               const uint8_t* cycle_start, double* Pmacro_out, gff_step_report* reports, gff_status* per_rve) {
    const int n = B.n;
    const StateLayout L(n);
    const int tangent = B.mixed ? TANGENT_F32 : TANGENT_F64;
    std::vector<gff_status> status(n, GFF_OK);
    int* hst = reinterpret_cast<int*>(B.h_pin + 64 * std::max(n, 4));  // pinned image of the state block
    for (int k = 0; k < nsteps; ++k) {
        const auto t0 = std::chrono::steady_clock::now();
        const double* Fb = Fbar + 9 * k;
        const uint8_t* mk = mask + 9 * k;
        const double* Pb = Pbar + 9 * k;
        if (cycle_start && cycle_start[k])
            for (int r = 0; r < n; ++r)
                if (status[r] == GFF_OK) BTRY(launch_fip_reset(B.h[r]));
        // zero-fluctuation start of every RVE, then the extrapolated warm start where asked for
        for (int r = 0; r < n; ++r) BTRY(launch_sum9(B.h[r]->d_F, B.h[r]->N, B.d_partial, B.d_out + 9 * r, B.st));
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        double add9[9];
        for (int c = 0; c < 9; ++c) add9[c] = mk[c] ? Pb[c] : 0.0;
        std::vector<double> Fsum(B.h_pin, B.h_pin + 9 * n);
        bool warm0[MAX_BATCH], nowarm[MAX_BATCH];
        std::vector<int> wused(n, 0);
        for (int r = 0; r < n; ++r) {
            gff_handle* h = B.h[r];
            for (int c = 0; c < 9; ++c) h->cur_d9[c] = mk[c] ? 0.0 : Fb[c] - Fsum[9 * r + c] / (double)h->N;
            warm0[r] = first_eval_warm(h, h->cur_d9);
            nowarm[r] = false;
            BTRY(launch_add_const9(h->d_Fk, h->d_F, h->cur_d9, h->N, B.st));
            if (status[r] == GFF_OK && h->opt.warm_start == GFF_WARM_EXTRAPOLATE) {
                cudaError_t e = warm_guess(nullptr, h, h->cur_d9, &wused[r]);
                if (e != cudaSuccess) return cuda_fail(B.h[0], e, "warm start");
            }
        }
        {
            gff_status st = set_residual_epilogue(B, add9);
            if (st != GFF_OK) return st;
        }
        // per-increment state, constitutive arguments (dt), then the increment's graph
        std::memset(hst, 0, sizeof(int) * L.total);
        for (int r = 0; r < n; ++r) {
            const bool in = status[r] == GFF_OK;
            hst[L.stat + r] = in ? ST_ACTIVE : ST_IDLE;
            hst[L.inactive + 2 * r] = in ? 0 : 1;
            hst[L.ksk + 2 * r] = 1;
        }
        BTRY(cudaMemcpyAsync(B.d_state, hst, sizeof(int) * L.total, cudaMemcpyHostToDevice, B.st));
        BTRY(upload_constitutive_batch(B.h, n, dt[k], tangent, warm0, B.d_state + L.warm, B.d_state + L.inactive,
                                       B.d_state + L.cpflag, B.d_cargsP, &B.blocksP, B.st));
        BTRY(upload_constitutive_batch(B.h, n, dt[k], tangent, nowarm, nullptr, B.d_state + L.ksk,
                                       B.d_state + L.kflag, B.d_cargsK, &B.blocksK, B.st));
        ProjArgs pa;
        pa.kind = B.h[0]->opt.projection;
        unsigned key = 0;
        for (int c = 0; c < 9; ++c) {
            pa.mask[c] = mk[c] ? 1.0f : 0.0f;
            key |= (mk[c] ? 1u : 0u) << c;
        }
        cudaGraphExec_t ex = nullptr;
        {
            gff_status st = increment_graph(B, pa, key, &ex);
            if (st != GFF_OK) return st;
        }
        BTRY(cudaGraphLaunch(ex, B.st));
        BTRY(cudaMemcpyAsync(hst, B.d_state, sizeof(int) * L.total, cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_dvals, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        std::vector<double> resv(B.h_pin, B.h_pin + n), resfirst(B.h_pin + n, B.h_pin + 2 * n);
        // commit the RVEs converged in the batch; redo the failed ones on their own handles
        std::vector<gff_step_report> rep(n);
        for (int r = 0; r < n; ++r) {
            std::memset(&rep[r], 0, sizeof(gff_step_report));
            if (status[r] != GFF_OK) continue;
            gff_handle* h = B.h[r];
            if (hst[L.stat + r] == ST_DONE) {
                gff_status sc = commit_rve(B, r, &Fsum[9 * r]);
                if (sc != GFF_OK) return sc;
                rep[r].newton_iters = hst[L.newton + r];
                rep[r].cg_iters = hst[L.cgsum + r];
                rep[r].residual = resv[r];
                rep[r].residual_first = resfirst[r];
                rep[r].warm_start_used = wused[r];
            } else {
                h->err.clear();
                const gff_status sf = gff_step(h, dt[k], Fb, mk, Pb, &rep[r]);
                if (sf != GFF_OK) status[r] = sf;
            }
        }
        for (int r = 0; r < n; ++r)
            if (status[r] == GFF_OK) {
                BTRY(launch_sum9(B.h[r]->d_P, B.h[r]->N, B.d_partial, B.d_out + 18 * r, B.st));
                BTRY(launch_sum9(B.h[r]->d_F, B.h[r]->N, B.d_partial, B.d_out + 18 * r + 9, B.st));
            }
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 18 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int r = 0; r < n; ++r) {
            gff_step_report& rp = rep[r];
            rp.seconds = secs;
            if (status[r] == GFF_OK)
                for (int c = 0; c < 9; ++c) {
                    rp.Pmacro[c] = B.h_pin[18 * r + c] / (double)B.h[r]->N;
                    rp.Fmacro[c] = B.h_pin[18 * r + 9 + c] / (double)B.h[r]->N;
                }
            if (status[r] == GFF_OK) {
                for (int c = 0; c < 9; ++c) B.h[r]->Pmacro_committed[c] = rp.Pmacro[c];
            }
            if (reports) reports[(size_t)r * nsteps + k] = rp;
            if (Pmacro_out) std::memcpy(Pmacro_out + ((size_t)r * nsteps + k) * 9, rp.Pmacro, 9 * sizeof(double));
        }
    }
    gff_status first = GFF_OK;
    for (int r = 0; r < n; ++r) {
        if (per_rve) per_rve[r] = status[r];
        if (first == GFF_OK) first = status[r];
    }
    return first;
}

}  // namespace

__attribute__((visibility("default"))) gff_status gff_batch_run(int n, gff_handle* const* hs, int nsteps,
                                                                const double* dt, const double* Fbar,
                                                                const uint8_t* mask, const double* Pbar,
                                                                const uint8_t* cycle_start, double* Pmacro_out,
                                                                gff_step_report* reports, gff_status* per_rve) {
    if (n < 1 || n > MAX_BATCH || !hs || nsteps < 0 || !dt || !Fbar || !mask || !Pbar) return GFF_ERR_ARG;
    for (int r = 0; r < n; ++r) {
        if (!hs[r]) return GFF_ERR_ARG;
        for (int q = 0; q < r; ++q)
            if (hs[q] == hs[r]) return GFF_ERR_ARG;
        if (hs[r]->small_strain) {
            set_error(hs[0], "batch: the small-strain variant runs one handle at a time (gff_run_history)");
            return GFF_ERR_ARG;
        }
        const gff_options& a = hs[0]->opt;
        const gff_options& b = hs[r]->opt;
        if (hs[r]->device != hs[0]->device || a.precision != b.precision || a.projection != b.projection ||
            a.newton_tol != b.newton_tol || a.cg_tol != b.cg_tol || a.newton_max != b.newton_max ||
            a.cg_max != b.cg_max) {
            set_error(hs[0], "batch: handles differ in device or options");
            return GFF_ERR_ARG;
        }
    }
    for (int k = 0; k < nsteps; ++k)
        if (!(dt[k] > 0)) return GFF_ERR_ARG;
    for (int r = 0; r < n; ++r) {
        gff_status st = prepare_for_increments(hs[r]);
        if (st != GFF_OK) {
            if (per_rve) per_rve[r] = st;
            return st;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return GFF_ERR_CUDA;
    Batch B;
    B.n = n;
    for (int r = 0; r < n; ++r) {
        B.h[r] = hs[r];
        B.saved[r] = hs[r]->stream;
    }
    if (cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking) != cudaSuccess) return GFF_ERR_CUDA;
    for (int r = 0; r < n; ++r) hs[r]->stream = B.st;  // per-RVE helper launches join the batch stream
    gff_status st = setup(B);
    if (st == GFF_OK) st = run(B, nsteps, dt, Fbar, mask, Pbar, cycle_start, Pmacro_out, reports, per_rve);
    if (cudaStreamSynchronize(B.st) != cudaSuccess && st == GFF_OK) st = GFF_ERR_CUDA;
    return st;
}
