// Batched increments of several RVEs of different sizes (gff_batch_run).
//
// All RVEs follow one macroscopic loading history.  Every per-iteration step
// of the Newton-CG loop (Sect. 2.1) is one launch over all RVEs: the
// constitutive update, the residual projection, the norms, and each CG
// iteration (three apply kernels + the CG vector kernels).  A block finds its
// RVE in a prefix table of the launch; per-RVE CG scalars and stop flags live
// on the device, so RVEs converge independently and a finished RVE's blocks
// return at entry.  The CG iterations run in chunks of CG_CHUNK; the chunk is
// captured once into a CUDA graph and replayed, the host reading the stop
// flags once per chunk.  Each RVE's arithmetic (including every reduction's
// block structure) is exactly that of gff_step on its own handle, so the
// batched result equals the one-by-one result bit for bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "gff_internal.cuh"

using namespace gff;

namespace {

constexpr int CG_CHUNK = 8;

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

struct Batch {
    int n = 0;
    cudaStream_t st = nullptr;
    cudaStream_t saved[MAX_BATCH];
    gff_handle* h[MAX_BATCH];
    bool mixed = false;
    // device arena
    DevBuf arena;
    RveApply* d_res = nullptr;
    RveApply* d_cgapply = nullptr;
    RveVec* d_vec = nullptr;     // CG vectors in the solve precision
    RveVec* d_nb = nullptr;      // (b, b): residual norms
    RveVec* d_nP = nullptr;      // (P, P)
    RveVec* d_nr32 = nullptr;    // (r32, r32)
    int* d_start_pl = nullptr;
    int* d_start_zres = nullptr;
    int* d_start_zcg = nullptr;
    double* d_cg = nullptr;      // [n][8]
    int* d_cgflag = nullptr;     // [n][2]
    int* d_inactive = nullptr;   // [n][2] (stride 2 like the CG flags)
    int* d_cpflag = nullptr;     // [n]
    double* d_partial = nullptr; // [max(n, 9)][RED_BLOCKS]
    double* d_out = nullptr;     // [18 n]
    double* d_rr0 = nullptr;     // [n][2]
    void* d_cscratch = nullptr;
    // pinned host mirror
    double* h_pin = nullptr;
    BatchLaunch bl_res{}, bl_cg{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool no_graph = false;

    ~Batch() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (h_pin) cudaFreeHost(h_pin);
        for (int r = 0; r < n; ++r) h[r]->stream = saved[r];
        if (st) cudaStreamDestroy(st);
    }
};

gff_status cuda_fail(gff_handle* h, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "batch %s: %s", what, cudaGetErrorString(e));
    set_error(h, buf);
    return GFF_ERR_CUDA;
}

#define BTRY(expr)                                              \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return cuda_fail(B.h[0], e_, #expr); \
    } while (0)

template <typename T> bool vec_aligned(const GridDev& g, const void* p) {
    return (g.nx % (16 / (int)sizeof(T))) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// Launch description of a batched apply over `rv` for precision T.
template <typename T>
BatchLaunch make_launch(Batch& B, const std::vector<RveApply>& rv, RveApply* d_rv, int* d_start_z, const Tune& tn,
                        bool withK, std::vector<int>& start_pl, std::vector<int>& start_z) {
    BatchLaunch bl{};
    bl.n = B.n;
    bl.rv = d_rv;
    bl.tn = tn;
    // the batched passes run the one-block-per-strip z kernel (at most 256 threads)
    // and the one-block-per-plane inverse (at most 512): the thread counts of the
    // persistent variants (TMA z pass, streamed inverse) are mapped onto them.
    // Every launch shape gives the same bits, so the results do not change.
    bl.tn.t_z = std::min(bl.tn.t_z, 256);
    bl.tn.t_inv = std::min(bl.tn.t_inv, 512);
    bl.withK = withK;
    bl.vin = bl.vout = true;
    start_pl.assign(B.n + 1, 0);
    start_z.assign(B.n + 1, 0);
    for (int r = 0; r < B.n; ++r) {
        const GridDev& g = rv[r].g;
        start_pl[r + 1] = start_pl[r] + 9 * g.nz;
        start_z[r + 1] = start_z[r] + zproj_blocks(g, tn.wz);
        bl.smem_plane = std::max(bl.smem_plane, batch_plane_smem(g.nx, g.ny, (int)sizeof(typename C2<T>::t)));
        bl.smem_z = std::max(bl.smem_z, batch_z_smem<T>(g, tn.wz));
        bl.vin = bl.vin && vec_aligned<T>(g, rv[r].x) && (!withK || vec_aligned<T>(g, rv[r].K));
        bl.vout = bl.vout && vec_aligned<T>(g, rv[r].y);
    }
    bl.start_plane = B.d_start_pl;
    bl.start_z = d_start_z;
    bl.blocks_plane = start_pl[B.n];
    bl.blocks_z = start_z[B.n];
    return bl;
}

// One CG iteration for all RVEs (apply + alpha + update/beta/direction).
template <typename T>
cudaError_t cg_iteration(Batch& B, const ProjArgs& pa) {
    cudaError_t e = launch_galerkin_batch<T>(B.bl_cg, pa, B.st);
    if (e == cudaSuccess) e = launch_cg_alpha_batch<T>(B.n, B.d_vec, B.d_partial, B.d_cg, B.d_cgflag, B.st);
    if (e == cudaSuccess) e = launch_cg_step_batch<T>(B.n, B.d_vec, B.d_partial, B.d_cg, B.d_cgflag, B.st);
    return e;
}

// CG for every RVE with rr0 >= 0 (rr0 < 0: RVE not solving).  iters[r] out.
template <typename T>
gff_status cg_batch(Batch& B, const ProjArgs& pa, const double* rr0, const double* stop, int cg_max, int* iters,
                    bool* breakdown) {
    const int n = B.n;
    for (int r = 0; r < n; ++r) {
        B.h_pin[2 * r] = rr0[r];
        B.h_pin[2 * r + 1] = stop[r] * stop[r];
    }
    BTRY(cudaMemcpyAsync(B.d_rr0, B.h_pin, 2 * n * sizeof(double), cudaMemcpyHostToDevice, B.st));
    BTRY(launch_cg_init_batch(n, B.d_cg, B.d_cgflag, B.d_rr0, B.st));
    int done = 0;
    std::vector<int> fl(2 * n);
    while (done < cg_max) {
        const int k = std::min(CG_CHUNK, cg_max - done);
        if (k == CG_CHUNK && B.gexec) {
            BTRY(cudaGraphLaunch(B.gexec, B.st));
        } else if (k == CG_CHUNK && done > 0 && !B.no_graph) {
            // first full chunk after an eager one: capture it (kernel attributes are already set)
            BTRY(cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < CG_CHUNK && e == cudaSuccess; ++i) e = cg_iteration<T>(B, pa);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(B.st, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&B.gexec, g, 0);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                // capture not possible here: keep launching the chunk directly
                if (g) cudaGraphDestroy(g);
                B.gexec = nullptr;
                B.no_graph = true;
                cudaGetLastError();
                for (int i = 0; i < k; ++i) BTRY(cg_iteration<T>(B, pa));
            } else {
                B.graph = g;
                BTRY(cudaGraphLaunch(B.gexec, B.st));
            }
        } else {
            for (int i = 0; i < k; ++i) BTRY(cg_iteration<T>(B, pa));
        }
        done += k;
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_cgflag, 2 * n * sizeof(int), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        std::memcpy(fl.data(), B.h_pin, 2 * n * sizeof(int));
        bool all = true;
        for (int r = 0; r < n; ++r) all = all && fl[2 * r] != 0;
        if (all) break;
    }
    BTRY(cudaMemcpyAsync(B.h_pin, B.d_cg, 8 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
    BTRY(cudaMemcpyAsync(B.h_pin + 8 * n, B.d_cgflag, 2 * n * sizeof(int), cudaMemcpyDeviceToHost, B.st));
    BTRY(cudaStreamSynchronize(B.st));
    std::memcpy(fl.data(), B.h_pin + 8 * n, 2 * n * sizeof(int));
    for (int r = 0; r < n; ++r) {
        iters[r] = (int)B.h_pin[8 * r + CG_ITERS];
        breakdown[r] = fl[2 * r + 1] != 0;
    }
    return GFF_OK;
}

gff_status setup(Batch& B) {
    const int n = B.n;
    const gff_options& o = B.h[0]->opt;
    B.mixed = o.precision == GFF_PREC_MIXED;
    // arena
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t a = off;
        off += (bytes + 255) / 256 * 256;
        return a;
    };
    const size_t o_res = take(sizeof(RveApply) * n), o_cga = take(sizeof(RveApply) * n);
    const size_t o_vec = take(sizeof(RveVec) * n), o_nb = take(sizeof(RveVec) * n), o_nP = take(sizeof(RveVec) * n);
    const size_t o_nr32 = take(sizeof(RveVec) * n);
    const size_t o_spl = take(sizeof(int) * (n + 1)), o_szr = take(sizeof(int) * (n + 1));
    const size_t o_szc = take(sizeof(int) * (n + 1));
    const size_t o_cg = take(sizeof(double) * 8 * n), o_cgf = take(sizeof(int) * 2 * n);
    const size_t o_ina = take(sizeof(int) * 2 * n), o_cpf = take(sizeof(int) * n);
    // partial sums: n RVEs x RED_BLOCKS (batched dots) or 9 x RED_BLOCKS (per-component sums)
    const size_t o_part = take(sizeof(double) * RED_BLOCKS * std::max(n, 9));
    const size_t o_out = take(sizeof(double) * 18 * n);
    const size_t o_rr0 = take(sizeof(double) * 2 * n), o_cs = take(constitutive_batch_scratch_bytes());
    BTRY(cudaMalloc(&B.arena.p, off));
    unsigned char* d = static_cast<unsigned char*>(B.arena.p);
    B.d_res = reinterpret_cast<RveApply*>(d + o_res);
    B.d_cgapply = reinterpret_cast<RveApply*>(d + o_cga);
    B.d_vec = reinterpret_cast<RveVec*>(d + o_vec);
    B.d_nb = reinterpret_cast<RveVec*>(d + o_nb);
    B.d_nP = reinterpret_cast<RveVec*>(d + o_nP);
    B.d_nr32 = reinterpret_cast<RveVec*>(d + o_nr32);
    B.d_start_pl = reinterpret_cast<int*>(d + o_spl);
    B.d_start_zres = reinterpret_cast<int*>(d + o_szr);
    B.d_start_zcg = reinterpret_cast<int*>(d + o_szc);
    B.d_cg = reinterpret_cast<double*>(d + o_cg);
    B.d_cgflag = reinterpret_cast<int*>(d + o_cgf);
    B.d_inactive = reinterpret_cast<int*>(d + o_ina);
    B.d_cpflag = reinterpret_cast<int*>(d + o_cpf);
    B.d_partial = reinterpret_cast<double*>(d + o_part);
    B.d_out = reinterpret_cast<double*>(d + o_out);
    B.d_rr0 = reinterpret_cast<double*>(d + o_rr0);
    B.d_cscratch = d + o_cs;
    BTRY(cudaMallocHost(&B.h_pin, sizeof(double) * 64 * std::max(n, 4)));

    // descriptors
    std::vector<RveApply> res(n), cga(n);
    std::vector<RveVec> vec(n), nb(n), nP(n), nr32(n);
    int big = 0;
    for (int r = 0; r < n; ++r)
        if (B.h[r]->N > B.h[big]->N) big = r;
    for (int r = 0; r < n; ++r) {
        gff_handle* h = B.h[r];
        res[r].g = h->g;
        res[r].x = h->d_P;
        res[r].K = nullptr;
        res[r].y = h->d_b;
        res[r].spec = h->d_spec;
        res[r].skip = B.d_inactive + 2 * r;
        cga[r].g = h->g;
        cga[r].spec = h->d_spec;
        cga[r].oa.scale = 1.0 / (double)h->N;
        for (int c = 0; c < 9; ++c) cga[r].oa.add[c] = 0.0;
        cga[r].skip = B.d_cgflag + 2 * r;
        const long long n9 = 9 * h->N;
        if (B.mixed) {
            cga[r].x = h->d_p32;
            cga[r].K = h->d_K32;
            cga[r].y = h->d_Ap32;
            vec[r] = {h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, n9};
        } else {
            cga[r].x = h->d_p;
            cga[r].K = h->d_K;
            cga[r].y = h->d_Ap;
            vec[r] = {h->d_x, h->d_r, h->d_p, h->d_Ap, n9};
        }
        nb[r] = {h->d_b, h->d_b, nullptr, nullptr, n9};
        nP[r] = {h->d_P, h->d_P, nullptr, nullptr, n9};
        nr32[r] = {h->d_r32, h->d_r32, nullptr, nullptr, n9};
    }
    std::vector<int> spl, szr, szc;
    B.bl_res = make_launch<double>(B, res, B.d_res, B.d_start_zres, B.h[big]->tune[0], false, spl, szr);
    if (B.mixed)
        B.bl_cg = make_launch<float>(B, cga, B.d_cgapply, B.d_start_zcg, B.h[big]->tune[1], true, spl, szc);
    else
        B.bl_cg = make_launch<double>(B, cga, B.d_cgapply, B.d_start_zcg, B.h[big]->tune[0], true, spl, szc);
    BTRY(cudaMemcpyAsync(B.d_res, res.data(), sizeof(RveApply) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_cgapply, cga.data(), sizeof(RveApply) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_vec, vec.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nb, nb.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nP, nP.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_nr32, nr32.data(), sizeof(RveVec) * n, cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_start_pl, spl.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_start_zres, szr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaMemcpyAsync(B.d_start_zcg, szc.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaStreamSynchronize(B.st));  // the host vectors above go out of scope
    return GFF_OK;
}

// Output epilogue of the residual projection b = -G_M(P) + M : Pbar: -1/N
// and the mask term; set once per increment (Pbar and the mask may change).
gff_status set_residual_epilogue(Batch& B, const double* add9) {
    std::vector<OutArgs> oa(B.n);
    for (int r = 0; r < B.n; ++r) {
        oa[r].scale = -1.0 / (double)B.h[r]->N;
        for (int c = 0; c < 9; ++c) oa[r].add[c] = add9[c];
    }
    for (int r = 0; r < B.n; ++r)
        BTRY(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(B.d_res + r) + offsetof(RveApply, oa), &oa[r],
                             sizeof(OutArgs), cudaMemcpyHostToDevice, B.st));
    BTRY(cudaStreamSynchronize(B.st));
    return GFF_OK;
}

gff_status run(Batch& B, int nsteps, const double* dt, const double* Fbar, const uint8_t* mask, const double* Pbar,
               const uint8_t* cycle_start, double* Pmacro_out, gff_step_report* reports, gff_status* per_rve) {
    const int n = B.n;
    const gff_options& o = B.h[0]->opt;
    std::vector<gff_status> status(n, GFF_OK);
    for (int k = 0; k < nsteps; ++k) {
        const auto t0 = std::chrono::steady_clock::now();
        const double* Fb = Fbar + 9 * k;
        const uint8_t* mk = mask + 9 * k;
        const double* Pb = Pbar + 9 * k;
        if (cycle_start && cycle_start[k])
            for (int r = 0; r < n; ++r)
                if (status[r] == GFF_OK) BTRY(launch_fip_reset(B.h[r]));
        // zero-fluctuation start of every RVE
        for (int r = 0; r < n; ++r) BTRY(launch_sum9(B.h[r]->d_F, B.h[r]->N, B.d_partial, B.d_out + 9 * r, B.st));
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        double add9[9];
        for (int c = 0; c < 9; ++c) add9[c] = mk[c] ? Pb[c] : 0.0;
        // per RVE: mean F of the committed state, prescribed change, warm first return maps (as gff_step)
        std::vector<double> Fold(9 * n);
        std::vector<char> warm0(n);
        for (int r = 0; r < n; ++r) {
            gff_handle* h = B.h[r];
            for (int c = 0; c < 9; ++c) {
                Fold[9 * r + c] = B.h_pin[9 * r + c] / (double)h->N;
                h->cur_d9[c] = mk[c] ? 0.0 : Fb[c] - Fold[9 * r + c];
            }
            warm0[r] = first_eval_warm(h, h->cur_d9);
            BTRY(launch_add_const9(h->d_Fk, h->d_F, h->cur_d9, h->N, B.st));
        }
        {
            gff_status st = set_residual_epilogue(B, add9);
            if (st != GFF_OK) return st;
        }
        ProjArgs pa;
        pa.kind = o.projection;
        for (int c = 0; c < 9; ++c) pa.mask[c] = mk[c] ? 1.0f : 0.0f;
        std::vector<bool> active(n), conv(n, false);
        std::vector<int> newton(n, 0), cgsum(n, 0);
        std::vector<double> resv(n, 0.0);
        for (int r = 0; r < n; ++r) active[r] = status[r] == GFF_OK;
        for (int it = 0; it <= o.newton_max; ++it) {
            std::vector<int> ina(2 * n, 0);
            for (int r = 0; r < n; ++r) ina[2 * r] = active[r] ? 0 : 1;
            std::memcpy(B.h_pin, ina.data(), 2 * n * sizeof(int));
            BTRY(cudaMemcpyAsync(B.d_inactive, B.h_pin, 2 * n * sizeof(int), cudaMemcpyHostToDevice, B.st));
            BTRY(cudaMemsetAsync(B.d_cpflag, 0, n * sizeof(int), B.st));
            bool warm[MAX_BATCH];
            for (int r = 0; r < n; ++r) warm[r] = it > 0 || warm0[r];
            BTRY(launch_constitutive_batch(B.h, n, dt[k], B.mixed ? TANGENT_F32 : TANGENT_F64, warm, B.d_inactive,
                                           B.d_cpflag, B.d_cscratch, B.st, CONST_P));
            BTRY(launch_galerkin_batch<double>(B.bl_res, pa, B.st));
            gff_status st = GFF_OK;
            BTRY(launch_dot_batch<double>(n, B.d_nb, B.d_partial, B.d_out, B.st));
            BTRY(launch_dot_batch<double>(n, B.d_nP, B.d_partial, B.d_out + n, B.st));
            BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
            BTRY(cudaMemcpyAsync(B.h_pin + 2 * n, B.d_cpflag, n * sizeof(int), cudaMemcpyDeviceToHost, B.st));
            BTRY(cudaStreamSynchronize(B.st));
            std::vector<int> cpf(n);
            std::memcpy(cpf.data(), B.h_pin + 2 * n, n * sizeof(int));
            std::vector<double> rr0(n, -1.0), stop(n, 0.0);
            bool any = false;
            for (int r = 0; r < n; ++r) {
                if (!active[r]) continue;
                if (cpf[r]) {
                    status[r] = GFF_ERR_CP_FAIL;
                    active[r] = false;
                    continue;
                }
                const double nbv = std::sqrt(B.h_pin[r]), nPv = std::sqrt(B.h_pin[n + r]);
                resv[r] = nPv > 0 ? nbv / nPv : nbv;
                if (resv[r] <= o.newton_tol) {
                    conv[r] = true;
                    active[r] = false;
                    continue;
                }
                if (it == o.newton_max) {
                    status[r] = GFF_ERR_NO_CONVERGENCE;
                    active[r] = false;
                    continue;
                }
                rr0[r] = B.h_pin[r];
                stop[r] = std::fmax(o.cg_tol * nbv, 0.1 * o.newton_tol * nPv);
                any = true;
            }
            if (!any) break;
            // tangents of the RVEs that take a Newton correction (as gff_step: never at a converged iterate)
            {
                std::vector<int> inak(2 * n, 0);
                for (int r = 0; r < n; ++r) inak[2 * r] = rr0[r] >= 0 ? 0 : 1;
                std::memcpy(B.h_pin, inak.data(), 2 * n * sizeof(int));
                BTRY(cudaMemcpyAsync(B.d_inactive, B.h_pin, 2 * n * sizeof(int), cudaMemcpyHostToDevice, B.st));
                BTRY(cudaMemsetAsync(B.d_cpflag, 0, n * sizeof(int), B.st));
                bool nowarm[MAX_BATCH] = {false};
                BTRY(launch_constitutive_batch(B.h, n, dt[k], B.mixed ? TANGENT_F32 : TANGENT_F64, nowarm,
                                               B.d_inactive, B.d_cpflag, B.d_cscratch, B.st, CONST_K));
                BTRY(cudaMemcpyAsync(B.h_pin, B.d_cpflag, n * sizeof(int), cudaMemcpyDeviceToHost, B.st));
                BTRY(cudaStreamSynchronize(B.st));
                std::vector<int> kf(n);
                std::memcpy(kf.data(), B.h_pin, n * sizeof(int));
                for (int r = 0; r < n; ++r)
                    if (rr0[r] >= 0 && kf[r]) {
                        status[r] = GFF_ERR_CP_FAIL;
                        active[r] = false;
                        rr0[r] = -1.0;
                    }
            }
            // right-hand sides and starting vectors of the active RVEs
            for (int r = 0; r < n; ++r) {
                if (rr0[r] < 0) continue;
                gff_handle* h = B.h[r];
                const long long n9 = 9 * h->N;
                if (B.mixed) {
                    BTRY(launch_cast64to32(h->d_r32, h->d_b, n9, B.st));
                    BTRY(launch_zero<float>(h->d_x32, n9, B.st));
                    BTRY(cudaMemcpyAsync(h->d_p32, h->d_r32, n9 * sizeof(float), cudaMemcpyDeviceToDevice, B.st));
                } else {
                    BTRY(cudaMemcpyAsync(h->d_r, h->d_b, n9 * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
                    BTRY(launch_zero<double>(h->d_x, n9, B.st));
                    BTRY(cudaMemcpyAsync(h->d_p, h->d_r, n9 * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
                }
            }
            std::vector<int> its(n, 0);
            std::vector<char> bd(n, 0);
            bool* bdp = reinterpret_cast<bool*>(bd.data());
            if (B.mixed) {
                BTRY(launch_dot_batch<float>(n, B.d_nr32, B.d_partial, B.d_out, B.st));
                BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
                BTRY(cudaStreamSynchronize(B.st));
                for (int r = 0; r < n; ++r)
                    if (rr0[r] >= 0) rr0[r] = B.h_pin[r];
                st = cg_batch<float>(B, pa, rr0.data(), stop.data(), o.cg_max, its.data(), bdp);
            } else {
                st = cg_batch<double>(B, pa, rr0.data(), stop.data(), o.cg_max, its.data(), bdp);
            }
            if (st != GFF_OK) return st;
            for (int r = 0; r < n; ++r) {
                if (rr0[r] < 0) continue;
                gff_handle* h = B.h[r];
                if (bd[r]) {
                    status[r] = GFF_ERR_NO_CONVERGENCE;
                    active[r] = false;
                    continue;
                }
                if (B.mixed)
                    BTRY(launch_axpy_to64<float>(h->d_Fk, h->d_x32, 9 * h->N, B.st));
                else
                    BTRY(launch_axpy_to64<double>(h->d_Fk, h->d_x, 9 * h->N, B.st));
                cgsum[r] += its[r];
                ++newton[r];
            }
        }
        // commit the converged RVEs; the others keep their last committed state.  First the
        // increment history (mean F change, normalised fluctuation increment) as gff_step keeps it.
        for (int r = 0; r < n; ++r)
            if (conv[r]) BTRY(launch_sum9(B.h[r]->d_Fk, B.h[r]->N, B.d_partial, B.d_out + 9 * r, B.st));
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        for (int r = 0; r < n; ++r) {
            if (!conv[r]) continue;
            gff_handle* h = B.h[r];
            double dF[9];
            for (int c = 0; c < 9; ++c) dF[c] = B.h_pin[9 * r + c] / (double)h->N - Fold[9 * r + c];
            gff_status sh = record_history(h, h->cur_d9, dF, B.st);
            if (sh != GFF_OK) return sh;
        }
        for (int r = 0; r < n; ++r) {
            gff_handle* h = B.h[r];
            if (!conv[r] && status[r] == GFF_OK) status[r] = GFF_ERR_NO_CONVERGENCE;
            if (!conv[r]) continue;
            const long long N = h->N;
            BTRY(cudaMemcpyAsync(h->d_F, h->d_Fk, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
            if (h->any_cp) {
                BTRY(cudaMemcpyAsync(h->d_Fpi, h->d_Fpi_t, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
                BTRY(cudaMemcpyAsync(h->d_chi, h->d_chi_t, 12 * N * sizeof(double), cudaMemcpyDeviceToDevice, B.st));
                BTRY(launch_fip_accumulate(h));
            }
            h->K_valid = h->K32_valid = false;  // the converged iterate's tangent is not computed
            BTRY(launch_sum9(h->d_P, N, B.d_partial, B.d_out + 18 * r, B.st));
            BTRY(launch_sum9(h->d_F, N, B.d_partial, B.d_out + 18 * r + 9, B.st));
        }
        BTRY(cudaMemcpyAsync(B.h_pin, B.d_out, 18 * n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        BTRY(cudaStreamSynchronize(B.st));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int r = 0; r < n; ++r) {
            gff_step_report rep;
            std::memset(&rep, 0, sizeof rep);
            rep.newton_iters = newton[r];
            rep.cg_iters = cgsum[r];
            rep.residual = resv[r];
            rep.seconds = secs;
            if (conv[r])
                for (int c = 0; c < 9; ++c) {
                    rep.Pmacro[c] = B.h_pin[18 * r + c] / (double)B.h[r]->N;
                    rep.Fmacro[c] = B.h_pin[18 * r + 9 + c] / (double)B.h[r]->N;
                }
            if (reports) reports[(size_t)r * nsteps + k] = rep;
            if (Pmacro_out) std::memcpy(Pmacro_out + ((size_t)r * nsteps + k) * 9, rep.Pmacro, 9 * sizeof(double));
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
