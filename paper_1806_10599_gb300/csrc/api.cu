// C ABI of libgff: handle lifetime, grid tables, microstructure set-up and the
// Newton-Raphson / conjugate-gradient increment driver (Sect. 2.1).
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "bulk_copy.cuh"
#include "gff_internal.cuh"

using namespace gff;

namespace {

#define GFF_TRY(expr)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return fail(h, GFF_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

gff_status fail(gff_handle* h, gff_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
gff_status fail(gff_handle* h, gff_status st, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

// ------------------------------------------------------------------ axis plans and tables
struct TableLayout {
    size_t tw64, tw32, posx, fqy, fqz, qt64, qt32, total;
};

TableLayout table_layout() {
    TableLayout t;
    size_t o = 0;
    t.tw64 = o; o += 3 * MAXN * sizeof(double2);
    t.tw32 = o; o += 3 * MAXN * sizeof(float2);
    t.posx = o; o += MAXN * sizeof(int);
    t.fqy = o; o += MAXN * sizeof(int);
    t.fqz = o; o += MAXN * sizeof(int);
    t.qt64 = o; o += 6 * MAXN * sizeof(double);
    t.qt32 = o; o += 6 * MAXN * sizeof(float);
    t.total = o;
    return t;
}

gff_status build_tables(gff_handle* h) {
    const int n3[3] = {h->grid.nx, h->grid.ny, h->grid.nz};
    AxisPlan* pl[3] = {&h->g.ax, &h->g.ay, &h->g.az};
    for (int a = 0; a < 3; ++a)
        if (!make_axis_plan(n3[a], *pl[a]))
            return fail(h, GFF_ERR_ARG, "grid axis %d: n = %d unsupported (even, 4..%d, factors 2,3,5)", a, n3[a], MAXN);
    const TableLayout L = table_layout();
    std::vector<unsigned char> host(L.total, 0);
    double2* tw64 = reinterpret_cast<double2*>(host.data() + L.tw64);
    float2* tw32 = reinterpret_cast<float2*>(host.data() + L.tw32);
    int* posx = reinterpret_cast<int*>(host.data() + L.posx);
    int* fqy = reinterpret_cast<int*>(host.data() + L.fqy);
    int* fqz = reinterpret_cast<int*>(host.data() + L.fqz);
    double* qt64 = reinterpret_cast<double*>(host.data() + L.qt64);
    float* qt32 = reinterpret_cast<float*>(host.data() + L.qt32);
    const double twopi = 6.283185307179586476925286766559;
    for (int a = 0; a < 3; ++a) {
        const int n = n3[a];
        const double Lj = h->grid.L[a];
        for (int k = 0; k < n; ++k) {
            const double th = twopi * k / n;
            tw64[a * MAXN + k] = make_double2(std::cos(th), -std::sin(th));
            tw32[a * MAXN + k] = make_float2((float)std::cos(th), (float)-std::sin(th));
            // wave-vector tables: q = 2 pi kappa / n, kappa = k (k < n/2) or k - n
            const int kappa = (2 * k < n) ? k : k - n;
            const double q = twopi * kappa / n;
            const bool nyq = (2 * k == n);
            const double qc = q * n / Lj;
            const double qd = nyq ? 0.0 : std::tan(0.5 * q) * n / Lj;
            qt64[(0 * 3 + a) * MAXN + k] = qc;
            qt64[(1 * 3 + a) * MAXN + k] = qd;
            qt32[(0 * 3 + a) * MAXN + k] = (float)qc;
            qt32[(1 * 3 + a) * MAXN + k] = (float)qd;
        }
    }
    for (int p = 0; p < h->grid.nx; ++p) posx[axis_freq_of_pos(p, h->g.ax)] = p;
    for (int p = 0; p < h->grid.ny; ++p) fqy[p] = axis_freq_of_pos(p, h->g.ay);
    for (int p = 0; p < h->grid.nz; ++p) fqz[p] = axis_freq_of_pos(p, h->g.az);
    cudaError_t e = cudaMalloc(&h->tables, L.total);
    if (e != cudaSuccess) return fail(h, GFF_ERR_OOM, "tables: %s", cudaGetErrorString(e));
    e = cudaMemcpy(h->tables, host.data(), L.total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "tables copy: %s", cudaGetErrorString(e));
    unsigned char* d = static_cast<unsigned char*>(h->tables);
    for (int a = 0; a < 3; ++a) {
        h->g.tw64[a] = reinterpret_cast<const double2*>(d + L.tw64) + a * MAXN;
        h->g.tw32[a] = reinterpret_cast<const float2*>(d + L.tw32) + a * MAXN;
        for (int kind = 0; kind < 2; ++kind) {
            h->g.qt64[kind][a] = reinterpret_cast<const double*>(d + L.qt64) + (kind * 3 + a) * MAXN;
            h->g.qt32[kind][a] = reinterpret_cast<const float*>(d + L.qt32) + (kind * 3 + a) * MAXN;
        }
    }
    h->g.posx = reinterpret_cast<const int*>(d + L.posx);
    h->g.fqy = reinterpret_cast<const int*>(d + L.fqy);
    h->g.fqz = reinterpret_cast<const int*>(d + L.fqz);
    return GFF_OK;
}

// ------------------------------------------------------------------ crystallography (host)
void quat_rot(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    const double n = std::sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

inline double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

void stiffness(const gff_material& m, const double* R, double* Cout) {
    double C[81];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double v;
                    if (m.kind == GFF_MAT_SVK_ISO || m.kind == GFF_MAT_NEOHOOKE) {
                        const double lam = m.E * m.nu / ((1 + m.nu) * (1 - 2 * m.nu));
                        const double mu = m.E / (2 * (1 + m.nu));
                        v = lam * kd(i, j) * kd(k, l) + mu * (kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k));
                    } else {
                        v = m.C12 * kd(i, j) * kd(k, l) + m.C44 * (kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k));
                        if (i == j && j == k && k == l) v += m.C11 - m.C12 - 2 * m.C44;
                    }
                    C[27 * i + 9 * j + 3 * k + l] = v;
                }
    if (m.kind == GFF_MAT_SVK_ISO || m.kind == GFF_MAT_NEOHOOKE) {  // isotropic: no rotation
        std::memcpy(Cout, C, sizeof C);
        return;
    }
    // C'_ijkl = R_ia R_jb R_kc R_ld C_abcd, done one index at a time
    double t1[81], t2[81];
    auto rot_index = [&](const double* in, double* out, int pos) {
        for (int q = 0; q < 81; ++q) {
            int idx[4] = {q / 27, (q / 9) % 3, (q / 3) % 3, q % 3};
            double s = 0;
            for (int a = 0; a < 3; ++a) {
                int j2[4] = {idx[0], idx[1], idx[2], idx[3]};
                j2[pos] = a;
                s += R[3 * idx[pos] + a] * in[27 * j2[0] + 9 * j2[1] + 3 * j2[2] + j2[3]];
            }
            out[q] = s;
        }
    };
    rot_index(C, t1, 0);
    rot_index(t1, t2, 1);
    rot_index(t2, t1, 2);
    rot_index(t1, Cout, 3);
}

// 12 octahedral systems: normals (111), (-111), (1-11), (11-1); for each the
// <110> directions orthogonal to it, in lexicographic order of the six <110>
// vectors whose first non-zero entry is positive.
void slip_systems(double s[12][3], double m[12][3]) {
    const int nrm[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    const int dirs[6][3] = {{0, 1, -1}, {0, 1, 1}, {1, -1, 0}, {1, 0, -1}, {1, 0, 1}, {1, 1, 0}};
    int a = 0;
    for (int p = 0; p < 4; ++p)
        for (int d = 0; d < 6; ++d) {
            const int dot = nrm[p][0] * dirs[d][0] + nrm[p][1] * dirs[d][1] + nrm[p][2] * dirs[d][2];
            if (dot != 0) continue;
            for (int k = 0; k < 3; ++k) {
                s[a][k] = dirs[d][k] / std::sqrt(2.0);
                m[a][k] = nrm[p][k] / std::sqrt(3.0);
            }
            ++a;
        }
}

}  // namespace

struct gff_hostdata {
    std::vector<double> quat;
    std::vector<int> phase;
};

namespace {

// Orthonormal basis of the symmetric traceless 3x3 tensors (Frobenius product).
void deviatoric_basis(double e[5][9]) {
    const double r2 = std::sqrt(0.5), r6 = std::sqrt(1.0 / 6.0);
    for (int i = 0; i < 5; ++i)
        for (int k = 0; k < 9; ++k) e[i][k] = 0.0;
    e[0][0] = r2, e[0][4] = -r2;                     // (E11 - E22) / sqrt 2
    e[1][0] = -r6, e[1][4] = -r6, e[1][8] = 2 * r6;  // (2 E33 - E11 - E22) / sqrt 6
    e[2][1] = e[2][3] = r2;                          // (E12 + E21) / sqrt 2
    e[3][2] = e[3][6] = r2;                          // (E13 + E31) / sqrt 2
    e[4][5] = e[4][7] = r2;                          // (E23 + E32) / sqrt 2
}

// out[0..59] = P [5][12], P_ia = e_i : sym(S0_a); out[60..84] = C5^-1 [5][5],
// C5_ij = e_i : C : e_j.  False if C5 is not invertible.
bool deviatoric_factors(const double* S0, const double* C, double* out) {
    double e[5][9];
    deviatoric_basis(e);
    for (int i = 0; i < 5; ++i)
        for (int a = 0; a < 12; ++a) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) v += e[i][3 * k + l] * 0.5 * (S0[9 * a + 3 * k + l] + S0[9 * a + 3 * l + k]);
            out[12 * i + a] = v;
        }
    double M[5][10];  // [C5 | I], Gauss-Jordan with partial pivoting
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double v = 0.0;
            for (int ij = 0; ij < 9; ++ij)
                for (int kl = 0; kl < 9; ++kl) v += e[i][ij] * C[9 * ij + kl] * e[j][kl];
            M[i][j] = v;
            M[i][5 + j] = i == j ? 1.0 : 0.0;
        }
    for (int k = 0; k < 5; ++k) {
        int p = k;
        for (int i = k + 1; i < 5; ++i)
            if (std::fabs(M[i][k]) > std::fabs(M[p][k])) p = i;
        if (!(std::fabs(M[p][k]) > 0.0)) return false;
        for (int j = 0; j < 10; ++j) std::swap(M[k][j], M[p][j]);
        const double inv = 1.0 / M[k][k];
        for (int j = 0; j < 10; ++j) M[k][j] *= inv;
        for (int i = 0; i < 5; ++i)
            if (i != k) {
                const double f = M[i][k];
                for (int j = 0; j < 10; ++j) M[i][j] -= f * M[k][j];
            }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) out[60 + 5 * i + j] = M[i][5 + j];
    return true;
}

gff_status upload_grains(gff_handle* h, const std::vector<double>& quat, const std::vector<int>& phase) {
    const int ng = h->ngrains;
    std::vector<double> C(81 * (size_t)ng), S0(GEO_STRIDE * (size_t)ng), nrmprm((36 + 5 + 144) * (size_t)ng);
    std::vector<int> kind(ng);
    double s[12][3], m[12][3];
    slip_systems(s, m);
    h->any_cp = false;
    for (int g = 0; g < ng; ++g) {
        const int ph = phase[g];
        if (ph < 0 || ph >= 8 || !h->mat_set[ph]) return fail(h, GFF_ERR_STATE, "grain %d: phase %d has no material", g, ph);
        const gff_material& mt = h->mat[ph];
        if (h->small_strain && mt.kind != GFF_MAT_SVK_CUBIC && mt.kind != GFF_MAT_SVK_ISO)
            return fail(h, GFF_ERR_ARG, "grain %d: the small-strain variant takes linear elastic phases only", g);
        double R[9];
        quat_rot(&quat[4 * (size_t)g], R);
        stiffness(mt, R, &C[81 * (size_t)g]);
        kind[g] = mt.kind;
        if (mt.kind == GFF_MAT_CP_FCC) h->any_cp = true;
        for (int a = 0; a < 12; ++a) {
            double sr[3], mr[3];
            for (int i = 0; i < 3; ++i) {
                sr[i] = R[3 * i] * s[a][0] + R[3 * i + 1] * s[a][1] + R[3 * i + 2] * s[a][2];
                mr[i] = R[3 * i] * m[a][0] + R[3 * i + 1] * m[a][1] + R[3 * i + 2] * m[a][2];
            }
            double* geo = &S0[GEO_STRIDE * (size_t)g];
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) geo[GEO_S0 + 9 * a + 3 * i + j] = sr[i] * mr[j];
                nrmprm[36 * (size_t)g + 3 * a + i] = mr[i];
                geo[GEO_DIR + 3 * a + i] = sr[i];
                if (a % 3 == 0) geo[GEO_NRM + a + i] = mr[i];  // plane a / 3: systems 3p .. 3p+2 share it
            }
        }
        {
            // Voigt stiffness: pairs 11, 22, 33, 23, 13, 12
            const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
            double* geo = &S0[GEO_STRIDE * (size_t)g];
            const double* Cg = &C[81 * (size_t)g];
            for (int I = 0; I < 6; ++I)
                for (int J = 0; J < 6; ++J)
                    geo[GEO_C6 + 6 * I + J] = Cg[9 * (3 * vi[I] + vj[I]) + 3 * vi[J] + vj[J]];
        }
        // factors of the small-strain slip interaction H = P^T C5 P (see cp_correction_lowrank)
        if (!deviatoric_factors(&S0[GEO_STRIDE * (size_t)g], &C[81 * (size_t)g], &nrmprm[41 * (size_t)ng + 144 * (size_t)g]))
            return fail(h, GFF_ERR_ARG, "grain %d: stiffness not positive definite on deviatoric strains", g);
        double* pr = &nrmprm[36 * (size_t)ng + 5 * (size_t)g];
        pr[0] = mt.gdot0;
        pr[1] = mt.p_exp;
        pr[2] = mt.tau0;
        pr[3] = mt.c_af;
        pr[4] = mt.d_af;
    }
    GFF_TRY(cudaMemcpy(h->d_C, C.data(), C.size() * sizeof(double), cudaMemcpyHostToDevice));
    GFF_TRY(cudaMemcpy(h->d_S0, S0.data(), S0.size() * sizeof(double), cudaMemcpyHostToDevice));
    {
        std::vector<float> g32(G32_STRIDE * (size_t)ng, 0.f);
        for (int g = 0; g < ng; ++g) {
            float* d = &g32[G32_STRIDE * (size_t)g];
            const double* geo = &S0[GEO_STRIDE * (size_t)g];
            for (int k = 0; k < 108; ++k) d[G32_S0 + k] = (float)geo[GEO_S0 + k];
            for (int k = 0; k < 81; ++k) d[G32_C + k] = (float)C[81 * (size_t)g + k];
            for (int k = 0; k < 36; ++k) d[G32_DIR + k] = (float)geo[GEO_DIR + k];
            for (int k = 0; k < 12; ++k) d[G32_NRM + k] = (float)geo[GEO_NRM + k];
            for (int k = 0; k < 36; ++k) d[G32_C6 + k] = (float)geo[GEO_C6 + k];
            for (int k = 0; k < 85; ++k) d[G32_PC + k] = (float)nrmprm[41 * (size_t)ng + 144 * (size_t)g + k];
        }
        GFF_TRY(cudaMemcpy(h->d_geo32, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    GFF_TRY(cudaMemcpy(h->d_nrm, nrmprm.data(), nrmprm.size() * sizeof(double), cudaMemcpyHostToDevice));
    GFF_TRY(cudaMemcpy(h->d_gkind, kind.data(), kind.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<float> gq(5 * (size_t)ng);
    for (int g = 0; g < ng; ++g) {
        const double* q = &quat[4 * (size_t)g];
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double sgn = q[0] < 0 ? -1.0 : 1.0;  // q and -q are one rotation: keep w >= 0
        for (int c = 0; c < 4; ++c) gq[5 * (size_t)g + c] = (float)(sgn * q[c] / qn);
        gq[5 * (size_t)g + 4] = (float)phase[g];
    }
    GFF_TRY(cudaMemcpy(h->d_gq, gq.data(), gq.size() * sizeof(float), cudaMemcpyHostToDevice));
    return GFF_OK;
}

gff_status ensure_grains(gff_handle* h);

template <typename T> void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

gff_status dalloc(gff_handle* h, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(h, GFF_ERR_OOM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
    return GFF_OK;
}

// Read one device double (synchronises the stream).
gff_status fetch(gff_handle* h, const double* d, int n, double* out) {
    GFF_TRY(cudaMemcpyAsync(h->h_scal, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    GFF_TRY(cudaStreamSynchronize(h->stream));
    std::memcpy(out, h->h_scal, n * sizeof(double));
    return GFF_OK;
}

ProjArgs proj_args(const gff_handle* h, const uint8_t* mask9) {
    ProjArgs pa;
    pa.kind = h->opt.projection;
    pa.sym = h->small_strain;
    for (int c = 0; c < 9; ++c) pa.mask[c] = (mask9 && mask9[c]) ? 1.0f : 0.0f;
    return pa;
}

OutArgs out_args(const gff_handle* h, double scale_sign, const double* add9) {
    OutArgs oa;
    oa.scale = scale_sign / (double)h->N;
    for (int c = 0; c < 9; ++c) oa.add[c] = add9 ? add9[c] : 0.0;
    return oa;
}

}  // namespace

// =================================================================== API
// Definitions take C linkage from their declarations in gff.h.
#define GFF_EXPORT __attribute__((visibility("default")))


GFF_EXPORT void gff_options_default(gff_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->projection = GFF_PROJ_CONTINUOUS;
    o->precision = GFF_PREC_FP64;
    o->newton_tol = 1e-8;
    o->cg_tol = 1e-8;
    o->newton_max = 30;
    o->cg_max = 2000;
    o->max_cuts = 4;
    o->warm_start = 0;
    o->fs_k = 0.5;
    o->fs_sigma_y = 153e6;
}

GFF_EXPORT const char* gff_last_error(const gff_handle* h) { return h ? h->err.c_str() : "null handle"; }

static gff_status check_options(gff_handle* h, const gff_options* o) {
    if (o->projection != GFF_PROJ_CONTINUOUS && o->projection != GFF_PROJ_DISCRETE)
        return fail(h, GFF_ERR_ARG, "projection %d", o->projection);
    if (o->precision != GFF_PREC_FP64 && o->precision != GFF_PREC_MIXED)
        return fail(h, GFF_ERR_ARG, "precision %d", o->precision);
    if (!(o->newton_tol > 0) || !(o->cg_tol > 0) || o->newton_max < 0 || o->cg_max < 1 || o->max_cuts < 0)
        return fail(h, GFF_ERR_ARG, "tolerances / caps out of range");
    if (o->warm_start < GFF_WARM_OFF || o->warm_start > GFF_WARM_EXTRAPOLATE)
        return fail(h, GFF_ERR_ARG, "warm_start must be 0, 1, 2 or 3");
    return GFF_OK;
}

GFF_EXPORT gff_status gff_create(const gff_grid* grid, const gff_options* opt, gff_handle** out) {
    if (!grid || !out) return GFF_ERR_ARG;
    *out = nullptr;
    gff_handle* h = new gff_handle();
    h->grid = *grid;
    gff_options_default(&h->opt);
    if (opt) h->opt = *opt;
    gff_status st = check_options(h, &h->opt);
    if (st != GFF_OK) {
        *out = h;
        return st;
    }
    for (int a = 0; a < 3; ++a)
        if (!(grid->L[a] > 0)) {
            *out = h;
            return fail(h, GFF_ERR_ARG, "box length L[%d] must be positive", a);
        }
    cudaGetDevice(&h->device);
    h->N = (long long)grid->nx * grid->ny * grid->nz;
    h->nxh = grid->nx / 2 + 1;
    h->g.nx = grid->nx;
    h->g.ny = grid->ny;
    h->g.nz = grid->nz;
    h->g.nxh = h->nxh;
    h->g.N = h->N;
    h->g.wait_cycles = BULK_WAIT_CYCLES;
    *out = h;
    if ((st = build_tables(h)) != GFF_OK) return st;
    const long long N = h->N;
    const size_t f64 = 9 * N * sizeof(double), f32 = 9 * N * sizeof(float);
    struct A { void** p; size_t b; const char* w; } allocs[] = {
        {(void**)&h->d_F, f64, "F"},        {(void**)&h->d_Fk, f64, "Fk"},
        {(void**)&h->d_P, f64, "P"},        {(void**)&h->d_K, 9 * f64, "K"},
        {(void**)&h->d_b, f64, "b"},        {(void**)&h->d_x, f64, "x"},
        {(void**)&h->d_r, f64, "r"},        {(void**)&h->d_p, f64, "p"},
        {(void**)&h->d_Ap, f64, "Ap"},      {(void**)&h->d_K32, 9 * f32, "K32"},
        {(void**)&h->d_b32, f32, "b32"},    {(void**)&h->d_x32, f32, "x32"},
        {(void**)&h->d_r32, f32, "r32"},    {(void**)&h->d_p32, f32, "p32"},
        {(void**)&h->d_Ap32, f32, "Ap32"},
        {(void**)&h->d_spec, 9 * (size_t)grid->nz * grid->ny * h->nxh * sizeof(double2), "spectrum"},
        {(void**)&h->d_Fpi, f64, "Fpi"},    {(void**)&h->d_chi, 12 * N * sizeof(double), "chi"},
        {(void**)&h->d_Fpi_t, f64, "Fpi_t"}, {(void**)&h->d_chi_t, 12 * N * sizeof(double), "chi_t"},
        {(void**)&h->d_dg, 12 * N * sizeof(double), "dg"}, {(void**)&h->d_tau, 12 * N * sizeof(double), "tau"},
        {(void**)&h->d_acc, NACC * N * sizeof(double), "fip"}, {(void**)&h->d_flag, 32, "flag"},
        {(void**)&h->d_red, 32 * RED_BLOCKS * sizeof(double), "reduce"},
        {(void**)&h->d_scal, 64 * sizeof(double), "scalars"},
        {(void**)&h->d_gid, N * sizeof(int), "grain id"},
        {(void**)&h->d_yhist, 2 * f32, "increment history"},
    };
    for (auto& a : allocs)
        if ((st = dalloc(h, a.p, a.b, a.w)) != GFF_OK) return st;
    cudaError_t e = cudaMallocHost(&h->h_scal, 64 * sizeof(double));
    if (e != cudaSuccess) return fail(h, GFF_ERR_OOM, "pinned scalars: %s", cudaGetErrorString(e));
    return GFF_OK;
}

GFF_EXPORT void gff_destroy(gff_handle* h) {
    if (!h) return;
    cudaFree(h->tables);
    dfree(h->d_gid); dfree(h->d_C); dfree(h->d_S0); dfree(h->d_nrm); dfree(h->d_gkind); dfree(h->d_gphase);
    dfree(h->d_F); dfree(h->d_Fk); dfree(h->d_P); dfree(h->d_K); dfree(h->d_b); dfree(h->d_x); dfree(h->d_r);
    dfree(h->d_p); dfree(h->d_Ap); dfree(h->d_K32); dfree(h->d_b32); dfree(h->d_x32); dfree(h->d_r32);
    dfree(h->d_p32); dfree(h->d_Ap32); dfree(h->d_spec); dfree(h->d_Fpi); dfree(h->d_chi); dfree(h->d_Fpi_t);
    dfree(h->d_chi_t); dfree(h->d_dg); dfree(h->d_tau); dfree(h->d_acc); dfree(h->d_flag); dfree(h->d_red);
    dfree(h->d_scal); dfree(h->d_gq); dfree(h->d_yhist); dfree(h->d_geo32);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    for (int i = 0; i < h->pipe_nev; ++i) cudaEventDestroy(h->pipe_ev[i]);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete reinterpret_cast<gff_hostdata*>(h->hostdata);
    delete h;
}

GFF_EXPORT gff_status gff_set_stream(gff_handle* h, void* stream) {
    if (!h) return GFF_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_options(gff_handle* h, const gff_options* opt) {
    if (!h || !opt) return GFF_ERR_ARG;
    gff_status st = check_options(h, opt);
    if (st != GFF_OK) return st;
    h->opt = *opt;
    return GFF_OK;
}

static gff_status reset_state(gff_handle* h) {
    const long long N = h->N;
    std::vector<double> eye(9 * N);
    for (int c = 0; c < 9; ++c)
        for (long long v = 0; v < N; ++v) eye[c * N + v] = (c % 4 == 0) ? 1.0 : 0.0;
    // finite strain starts at F = I, the small-strain variant at eps = 0
    if (h->small_strain) {
        GFF_TRY(cudaMemset(h->d_F, 0, 9 * N * sizeof(double)));
        GFF_TRY(cudaMemset(h->d_Fk, 0, 9 * N * sizeof(double)));
    } else {
        GFF_TRY(cudaMemcpy(h->d_F, eye.data(), 9 * N * sizeof(double), cudaMemcpyHostToDevice));
        GFF_TRY(cudaMemcpy(h->d_Fk, eye.data(), 9 * N * sizeof(double), cudaMemcpyHostToDevice));
    }
    GFF_TRY(cudaMemcpy(h->d_Fpi, eye.data(), 9 * N * sizeof(double), cudaMemcpyHostToDevice));
    GFF_TRY(cudaMemset(h->d_chi, 0, 12 * N * sizeof(double)));
    GFF_TRY(cudaMemset(h->d_P, 0, 9 * N * sizeof(double)));
    GFF_TRY(cudaMemset(h->d_acc, 0, NACC * N * sizeof(double)));
    GFF_TRY(cudaMemset(h->d_flag, 0, 32));
    GFF_TRY(launch_fip_reset(h));
    GFF_TRY(cudaDeviceSynchronize());
    h->K_valid = h->K32_valid = false;
    h->nhist = 0;
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_microstructure(gff_handle* h, const int32_t* grain_id, int ngrains, const double* quat,
                                  const int32_t* grain_phase) {
    if (!h || !grain_id || !quat || !grain_phase || ngrains < 1) return fail(h, GFF_ERR_ARG, "bad microstructure args");
    for (long long v = 0; v < h->N; ++v)
        if (grain_id[v] < 0 || grain_id[v] >= ngrains) return fail(h, GFF_ERR_ARG, "grain_id[%lld] out of range", v);
    for (int g = 0; g < ngrains; ++g)
        if (grain_phase[g] < 0 || grain_phase[g] >= 8) return fail(h, GFF_ERR_ARG, "grain_phase[%d] out of range", g);
    dfree(h->d_C); dfree(h->d_S0); dfree(h->d_nrm); dfree(h->d_gkind); dfree(h->d_gq); dfree(h->d_geo32);
    h->ngrains = ngrains;
    gff_status st;
    if ((st = dalloc(h, (void**)&h->d_C, 81 * (size_t)ngrains * sizeof(double), "C")) != GFF_OK) return st;
    if ((st = dalloc(h, (void**)&h->d_S0, GEO_STRIDE * (size_t)ngrains * sizeof(double), "slip geometry")) != GFF_OK)
        return st;
    if ((st = dalloc(h, (void**)&h->d_nrm, (41 + 144) * (size_t)ngrains * sizeof(double), "normals")) != GFF_OK)
        return st;
    if ((st = dalloc(h, (void**)&h->d_gkind, (size_t)ngrains * sizeof(int), "kind")) != GFF_OK) return st;
    if ((st = dalloc(h, (void**)&h->d_geo32, G32_STRIDE * (size_t)ngrains * sizeof(float), "FP32 slip geometry")) !=
        GFF_OK)
        return st;
    if ((st = dalloc(h, (void**)&h->d_gq, 5 * (size_t)ngrains * sizeof(float), "grain quaternions")) != GFF_OK)
        return st;
    GFF_TRY(cudaMemcpy(h->d_gid, grain_id, h->N * sizeof(int), cudaMemcpyHostToDevice));
    gff_hostdata* hd = reinterpret_cast<gff_hostdata*>(h->hostdata);
    if (!hd) {
        hd = new gff_hostdata();
        h->hostdata = hd;
    }
    hd->quat.assign(quat, quat + 4 * (size_t)ngrains);
    hd->phase.assign(grain_phase, grain_phase + ngrains);
    h->have_ms = true;
    h->grains_ready = false;
    return reset_state(h);
}

GFF_EXPORT gff_status gff_set_material(gff_handle* h, int phase, const gff_material* m) {
    if (!h || !m || phase < 0 || phase >= 8) return fail(h, GFF_ERR_ARG, "bad material args");
    if (m->kind < GFF_MAT_SVK_CUBIC || m->kind > GFF_MAT_NEOHOOKE) return fail(h, GFF_ERR_ARG, "material kind %d", m->kind);
    if ((m->kind == GFF_MAT_SVK_ISO || m->kind == GFF_MAT_NEOHOOKE) && !(m->E > 0 && m->nu > -1 && m->nu < 0.5))
        return fail(h, GFF_ERR_ARG, "isotropic constants out of range");
    if (m->kind == GFF_MAT_CP_FCC) {
        const double p = m->p_exp;
        if (!(p >= 1 && p <= 64 && p == std::floor(p)) || !(m->tau0 > 0) || !(m->gdot0 > 0) || m->d_af < 0)
            return fail(h, GFF_ERR_ARG, "crystal-plasticity constants out of range");
    }
    h->mat[phase] = *m;
    h->mat_set[phase] = true;
    h->grains_ready = false;
    return GFF_OK;
}

namespace {
gff_status ensure_grains(gff_handle* h) {
    if (!h->have_ms) return fail(h, GFF_ERR_STATE, "no microstructure set");
    if (h->grains_ready) return GFF_OK;
    gff_hostdata* hd = reinterpret_cast<gff_hostdata*>(h->hostdata);
    gff_status st = upload_grains(h, hd->quat, hd->phase);
    if (st == GFF_OK) h->grains_ready = true;
    return st;
}

int field_comps(int which) {
    switch (which) {
        case GFF_FIELD_F: case GFF_FIELD_P: case GFF_FIELD_FP_INV: return 9;
        case GFF_FIELD_K: return 81;
        case GFF_FIELD_CHI: case GFF_FIELD_GAMMA: case GFF_FIELD_WCYC: return 12;
        case GFF_FIELD_PCYC: return 1;
        default: return 0;
    }
}

double* field_ptr(gff_handle* h, int which) {
    switch (which) {
        case GFF_FIELD_F: return h->d_F;
        case GFF_FIELD_P: return h->d_P;
        case GFF_FIELD_K: return h->d_K;
        case GFF_FIELD_FP_INV: return h->d_Fpi;
        case GFF_FIELD_CHI: return h->d_chi;
        case GFF_FIELD_GAMMA: return h->d_acc + 13 * h->N;
        case GFF_FIELD_PCYC: return h->d_acc;
        case GFF_FIELD_WCYC: return h->d_acc + 1 * h->N;
        default: return nullptr;
    }
}
}  // namespace

GFF_EXPORT gff_status gff_set_field(gff_handle* h, int which, const double* host) {
    if (!h || !host) return fail(h, GFF_ERR_ARG, "bad args");
    if (!h->have_ms) return fail(h, GFF_ERR_STATE, "no microstructure set");
    const int nc = field_comps(which);
    double* d = field_ptr(h, which);
    if (!nc || !d) return fail(h, GFF_ERR_ARG, "field %d", which);
    GFF_TRY(cudaMemcpyAsync(d, host, nc * h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (which == GFF_FIELD_F)
        GFF_TRY(cudaMemcpyAsync(h->d_Fk, host, 9 * h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (which == GFF_FIELD_K) h->K_valid = true, h->K32_valid = false;
    GFF_TRY(cudaStreamSynchronize(h->stream));
    return GFF_OK;
}

GFF_EXPORT gff_status gff_get_field(gff_handle* h, int which, double* host) {
    if (!h || !host) return fail(h, GFF_ERR_ARG, "bad args");
    const int nc = field_comps(which);
    double* d = field_ptr(h, which);
    if (!nc || !d) return fail(h, GFF_ERR_ARG, "field %d", which);
    GFF_TRY(cudaMemcpyAsync(host, d, nc * h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    GFF_TRY(cudaStreamSynchronize(h->stream));
    return GFF_OK;
}

GFF_EXPORT gff_status gff_constitutive(gff_handle* h, double dt) {
    if (!h) return GFF_ERR_ARG;
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    GFF_TRY(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    GFF_TRY(launch_constitutive(h, h->d_Fk, dt, TANGENT_F64_AND_F32));
    int flag = 0;
    GFF_TRY(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    GFF_TRY(cudaStreamSynchronize(h->stream));
    h->K_valid = h->K32_valid = true;
    if (flag) return fail(h, GFF_ERR_CP_FAIL, "return map failed in %d voxels", flag);
    return GFF_OK;
}

// FP64 applies need the FP64 tangent; FP32 applies take K32 or round the FP64 one.
static bool tangent_ready(const gff_handle* h, int precision) {
    return precision == GFF_PREC_FP64 ? h->K_valid : (h->K32_valid || h->K_valid);
}

GFF_EXPORT gff_status gff_apply_operator(gff_handle* h, int precision, const uint8_t* mask9, const void* x_dev, void* y_dev) {
    if (!h || !x_dev || !y_dev || x_dev == y_dev) return fail(h, GFF_ERR_ARG, "bad apply args");
    if (!tangent_ready(h, precision)) return fail(h, GFF_ERR_STATE, "no tangent for this precision: call gff_constitutive");
    const ProjArgs pa = proj_args(h, mask9);
    const OutArgs oa = out_args(h, 1.0, nullptr);
    if (precision == GFF_PREC_FP64) {
        GFF_TRY(launch_galerkin<double>(h, (const double*)x_dev, h->d_K, (double*)y_dev, pa, oa, h->d_spec));
    } else if (precision == GFF_PREC_MIXED) {
        if (!h->K32_valid) {
            GFF_TRY(launch_cast64to32(h->d_K32, h->d_K, 81 * h->N, h->stream));
            h->K32_valid = true;
        }
        GFF_TRY(launch_galerkin<float>(h, (const float*)x_dev, h->d_K32, (float*)y_dev, pa, oa,
                                       reinterpret_cast<float2*>(h->d_spec)));
    } else {
        return fail(h, GFF_ERR_ARG, "precision %d", precision);
    }
    return GFF_OK;
}

GFF_EXPORT gff_status gff_apply_operator_timed(gff_handle* h, int precision, const uint8_t* mask9,
                                               const void* x_dev, void* y_dev, float* ms_out) {
    if (!h || !x_dev || !y_dev || x_dev == y_dev || !ms_out) return fail(h, GFF_ERR_ARG, "bad apply args");
    if (!tangent_ready(h, precision)) return fail(h, GFF_ERR_STATE, "no tangent for this precision: call gff_constitutive");
    if (precision != GFF_PREC_FP64 && precision != GFF_PREC_MIXED) return fail(h, GFF_ERR_ARG, "precision %d", precision);
    const ProjArgs pa = proj_args(h, mask9);
    const OutArgs oa = out_args(h, 1.0, nullptr);
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e == cudaSuccess && precision == GFF_PREC_MIXED && !h->K32_valid) {
        e = launch_cast64to32(h->d_K32, h->d_K, 81 * h->N, h->stream);
        if (e == cudaSuccess) h->K32_valid = true;
    }
    if (e == cudaSuccess) {
        if (precision == GFF_PREC_FP64)
            e = launch_galerkin<double>(h, (const double*)x_dev, h->d_K, (double*)y_dev, pa, oa, h->d_spec, ev);
        else
            e = launch_galerkin<float>(h, (const float*)x_dev, h->d_K32, (float*)y_dev, pa, oa,
                                       reinterpret_cast<float2*>(h->d_spec), ev);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms_out[i], ev[i], ev[i + 1]);
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "timed apply: %s", cudaGetErrorString(e));
    return gff_sync(h);
}

GFF_EXPORT gff_status gff_apply_operator_host(gff_handle* h, int precision, const uint8_t* mask9, const void* x_host,
                                              void* y_host) {
    if (!h || !x_host || !y_host) return fail(h, GFF_ERR_ARG, "bad apply args");
    if (precision != GFF_PREC_FP64 && precision != GFF_PREC_MIXED) return fail(h, GFF_ERR_ARG, "precision %d", precision);
    if (!tangent_ready(h, precision)) return fail(h, GFF_ERR_STATE, "no tangent for this precision: call gff_constitutive");
    const ProjArgs pa = proj_args(h, mask9);
    const OutArgs oa = out_args(h, 1.0, nullptr);
    if (precision == GFF_PREC_FP64) {
        GFF_TRY(launch_galerkin_host<double>(h, (const double*)x_host, (double*)y_host, h->d_x, h->d_Ap, h->d_K, pa, oa,
                                             h->d_spec));
    } else {
        if (!h->K32_valid) {
            GFF_TRY(launch_cast64to32(h->d_K32, h->d_K, 81 * h->N, h->stream));
            h->K32_valid = true;
        }
        GFF_TRY(launch_galerkin_host<float>(h, (const float*)x_host, (float*)y_host, h->d_x32, h->d_Ap32, h->d_K32, pa,
                                            oa, reinterpret_cast<float2*>(h->d_spec)));
    }
    return gff_sync(h);
}

GFF_EXPORT gff_status gff_cg_kernels_timed(gff_handle* h, int precision, int reps, float* ms_out) {
    if (!h || !ms_out || reps < 1) return fail(h, GFF_ERR_ARG, "bad args");
    double* cg = h->d_scal + 32;
    int* flag = reinterpret_cast<int*>(h->d_scal + 48);
    cudaError_t e;
    if (precision == GFF_PREC_FP64)
        e = time_cg_kernels<double>(h->d_x, h->d_r, h->d_p, h->d_Ap, 9 * h->N, h->d_red, cg, flag, h->stream, reps,
                                    ms_out);
    else if (precision == GFF_PREC_MIXED)
        e = time_cg_kernels<float>(h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, 9 * h->N, h->d_red, cg, flag, h->stream,
                                   reps, ms_out);
    else
        return fail(h, GFF_ERR_ARG, "precision %d", precision);
    if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "timed CG kernels: %s", cudaGetErrorString(e));
    return GFF_OK;
}

GFF_EXPORT gff_status gff_measure_fp64_peak(double* gflops_out, double* ms_out) {
    if (!gflops_out) return GFF_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFF_ERR_CUDA;
    const int blocks = 4 * nsm;
    double* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) return GFF_ERR_OOM;
    float ms = 0.f;
    cudaError_t e = measure_fp64_fma(out, blocks, 8192, 5, nullptr, gflops_out, &ms);
    cudaFree(out);
    if (e != cudaSuccess) return GFF_ERR_CUDA;
    if (ms_out) *ms_out = ms;
    return GFF_OK;
}

GFF_EXPORT gff_status gff_sync(gff_handle* h) {
    if (!h) return GFF_ERR_ARG;
    int tmo = 0;
    GFF_TRY(cudaMemcpyAsync(h->h_scal, h->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    GFF_TRY(cudaStreamSynchronize(h->stream));
    std::memcpy(&tmo, h->h_scal, sizeof(int));
    if (tmo) {
        GFF_TRY(cudaMemsetAsync(h->d_flag + 2, 0, sizeof(int), h->stream));
        GFF_TRY(cudaStreamSynchronize(h->stream));
        return fail(h, GFF_ERR_TIMEOUT, "a bounded bulk-copy wait in an FFT pass gave up (%d)", tmo);
    }
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_wait_limit(gff_handle* h, long long cycles) {
    if (!h) return GFF_ERR_ARG;
    h->g.wait_cycles = cycles < 0 ? BULK_WAIT_CYCLES : cycles;
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_strain_measure(gff_handle* h, int mode) {
    if (!h || (mode != GFF_STRAIN_FINITE && mode != GFF_STRAIN_SMALL))
        return fail(h, GFF_ERR_ARG, "strain measure must be 0 or 1");
    h->small_strain = mode == GFF_STRAIN_SMALL ? 1 : 0;
    h->grains_ready = false;  // phases are checked against the variant again
    return h->have_ms ? reset_state(h) : GFF_OK;
}

GFF_EXPORT gff_status gff_set_return_map(gff_handle* h, int mode) {
    if (!h || mode < GFF_RETURN_MAP_DEFAULT || mode > GFF_RETURN_MAP_FP64)
        return fail(h, GFF_ERR_ARG, "return-map mode must be 0, 1, 2 or 3");
    h->cp_exact_only = mode == GFF_RETURN_MAP_EXACT ? 1 : 0;
    h->cp_f32_first = mode == GFF_RETURN_MAP_F32_FIRST ? 1 : (mode == GFF_RETURN_MAP_DEFAULT ? 2 : 0);
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_warm_start(gff_handle* h, gff_unet* u, int mode) {
    const bool net = mode == GFF_WARM_NET_IF_BETTER || mode == GFF_WARM_NET;
    if (!h || mode < GFF_WARM_OFF || mode > GFF_WARM_EXTRAPOLATE || (net && !u))
        return fail(h, GFF_ERR_ARG, "bad warm-start args");
    if (net && (h->grid.nx != h->grid.ny || h->grid.ny != h->grid.nz || h->grid.nx % 8))
        return fail(h, GFF_ERR_ARG, "the warm-start network needs a cubic grid with n divisible by 8");
    h->unet = net ? u : nullptr;
    h->opt.warm_start = mode;
    return GFF_OK;
}

GFF_EXPORT gff_status gff_set_tiles(gff_handle* h, const int* tiles) {
    if (!h || !tiles) return fail(h, GFF_ERR_ARG, "bad tiles args");
    Tune t[2];
    for (int p = 0; p < 2; ++p) {
        t[p].t_fwd = tiles[5 * p + 0];
        t[p].wz = tiles[5 * p + 1];
        t[p].t_z = tiles[5 * p + 2];
        t[p].t_inv = tiles[5 * p + 3];
        t[p].inv_blocks = tiles[5 * p + 4];
        t[p].z_blocks = tiles[10 + p];
    }
    if (!set_tiles(h, t[0], t[1])) return fail(h, GFF_ERR_ARG, "launch shapes not supported for this grid");
    GFF_TRY(preload_constitutive());
    return GFF_OK;
}

GFF_EXPORT gff_status gff_autotune(gff_handle* h, int* tiles_out) {
    if (!h) return GFF_ERR_ARG;
    GFF_TRY(autotune_galerkin(h));
    GFF_TRY(preload_constitutive());  // kernels loaded now, not inside the first increment
    if (tiles_out)
        for (int p = 0; p < 2; ++p) {
            tiles_out[5 * p + 0] = h->tune[p].t_fwd;
            tiles_out[5 * p + 1] = h->tune[p].wz;
            tiles_out[5 * p + 2] = h->tune[p].t_z;
            tiles_out[5 * p + 3] = h->tune[p].t_inv;
            tiles_out[5 * p + 4] = h->tune[p].inv_blocks;
            tiles_out[10 + p] = h->tune[p].z_blocks;
        }
    return GFF_OK;
}

GFF_EXPORT gff_status gff_project(gff_handle* h, int precision, const uint8_t* mask9, const void* x_dev, void* y_dev) {
    if (!h || !x_dev || !y_dev || x_dev == y_dev) return fail(h, GFF_ERR_ARG, "bad project args");
    const ProjArgs pa = proj_args(h, mask9);
    const OutArgs oa = out_args(h, 1.0, nullptr);
    if (precision == GFF_PREC_FP64) {
        GFF_TRY(launch_galerkin<double>(h, (const double*)x_dev, (const double*)nullptr, (double*)y_dev, pa, oa,
                                        h->d_spec));
    } else if (precision == GFF_PREC_MIXED) {
        GFF_TRY(launch_galerkin<float>(h, (const float*)x_dev, (const float*)nullptr, (float*)y_dev, pa, oa,
                                       reinterpret_cast<float2*>(h->d_spec)));
    } else {
        return fail(h, GFF_ERR_ARG, "precision %d", precision);
    }
    return GFF_OK;
}

// ------------------------------------------------------------------ Newton-CG increment
namespace {

// CG on G_M(K : dF) = b from dF = 0 (Sect. 2.1).  T = double: vectors
// d_x/d_r/d_p/d_Ap with K; T = float: the FP32 copies with K32.  Stops when
// ||r|| <= stop or after cg_max iterations.  The scalars (r.r, p.Ap, alpha,
// beta) and the stop test live on the device; the host launches iterations
// in chunks and reads the stop flag once per chunk.  Once the flag is set,
// every remaining kernel of the chunk returns at entry.
constexpr int CG_CHUNK = 8;

template <typename T>
gff_status cg_solve(gff_handle* h, const ProjArgs& pa, T* x, T* r, T* p, T* Ap, const T* K, double rr0, double stop,
                    int* iters) {
    const long long n = 9 * h->N;
    const OutArgs oa = out_args(h, 1.0, nullptr);
    typename C2<T>::t* spec = reinterpret_cast<typename C2<T>::t*>(h->d_spec);
    double* cg = h->d_scal + 32;
    int* flag = reinterpret_cast<int*>(h->d_scal + 48);
    GFF_TRY(launch_zero<T>(x, n, h->stream));
    GFF_TRY(cudaMemcpyAsync(p, r, n * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
    GFF_TRY(launch_cg_init(cg, flag, rr0, stop * stop, h->stream));
    int done = 0;
    int hflag[2] = {0, 0};
    while (done < h->opt.cg_max) {
        const int k = std::min(CG_CHUNK, h->opt.cg_max - done);
        for (int i = 0; i < k; ++i) {
            GFF_TRY(launch_galerkin<T>(h, p, K, Ap, pa, oa, spec, nullptr, flag));
            GFF_TRY(launch_cg_alpha<T>(p, Ap, n, h->d_red, cg, flag, h->stream));
            GFF_TRY(launch_cg_step<T>(x, r, p, Ap, n, h->d_red, cg, flag, h->stream));
        }
        done += k;
        GFF_TRY(cudaMemcpyAsync(h->h_scal, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        GFF_TRY(cudaStreamSynchronize(h->stream));
        std::memcpy(hflag, h->h_scal, sizeof hflag);
        if (hflag[0]) break;
    }
    double it_d;
    gff_status st = fetch(h, cg + CG_ITERS, 1, &it_d);
    if (st != GFF_OK) return st;
    *iters = (int)it_d;
    if (hflag[1]) return fail(h, GFF_ERR_NO_CONVERGENCE, "CG breakdown after %d iterations", *iters);
    return GFF_OK;
}

gff_status newton_increment(gff_handle* h, double dt, const double* Fbar, const uint8_t* mask, const double* Pbar,
                            gff_step_report* rep) {
    const long long N = h->N;
    const long long n = 9 * N;
    gff_status st;
    GFF_TRY(cudaMemsetAsync(h->d_flag + 2, 0, sizeof(int), h->stream));  // timeouts are counted per increment
    // zero-fluctuation start: F = F_{k-1} + dFbar on strain-controlled components
    double Fsum[9];
    GFF_TRY(launch_sum9(h->d_F, N, h->d_red, h->d_scal, h->stream));
    if ((st = fetch(h, h->d_scal, 9, Fsum)) != GFF_OK) return st;
    double d9[9], add9[9];
    for (int c = 0; c < 9; ++c) {
        d9[c] = mask[c] ? 0.0 : Fbar[c] - Fsum[c] / (double)N;
        add9[c] = mask[c] ? Pbar[c] : 0.0;
        h->cur_d9[c] = d9[c];
    }
    GFF_TRY(launch_add_const9(h->d_Fk, h->d_F, d9, N, h->stream));
    const ProjArgs pa = proj_args(h, mask);
    const OutArgs ores = out_args(h, -1.0, add9);
    const bool mixed = h->opt.precision == GFF_PREC_MIXED;
    int newton = 0, cgsum = 0;
    double res = 0.0, nb = 0.0, nP = 0.0, rr_b = 0.0;
    bool conv = false;
    double t_const = 0.0, t_res = 0.0, t_lin = 0.0, t_tan = 0.0;
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; ++i) GFF_TRY(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    int warm_used = 0, cp_fb = 0;
    double res_first = 0.0, cp_its = 0.0;
    // the report is written on every exit, failed attempts included (cut-back adds them up)
    struct RepGuard {
        gff_step_report* r;
        const int &newton, &cgsum, &warm_used, &cp_fb;
        const double &res, &t_const, &t_res, &t_lin, &res_first, &cp_its, &t_tan;
        ~RepGuard() {
            if (!r) return;
            r->newton_iters = newton;
            r->cg_iters = cgsum;
            r->residual = res;
            r->t_constitutive = t_const;
            r->t_residual = t_res;
            r->t_linear = t_lin;
            r->warm_start_used = warm_used;
            r->residual_first = res_first;
            r->cp_fallbacks = cp_fb;
            r->cp_local_iters = cp_its;
            r->t_tangent = t_tan;
        }
    } repg{rep, newton, cgsum, warm_used, cp_fb, res, t_const, t_res, t_lin, res_first, cp_its, t_tan};

    // P, K at d_Fk and the residual b = -G_M(P) + M : Pbar with its norms
    auto evaluate = [&](bool warm_dg) -> gff_status {
        GFF_TRY(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
        GFF_TRY(cudaMemsetAsync(h->d_flag + 4, 0, 2 * sizeof(int), h->stream));
        GFF_TRY(cudaEventRecord(ev[0], h->stream));
        GFF_TRY(launch_constitutive(h, h->d_Fk, dt, mixed ? TANGENT_F32 : TANGENT_F64, warm_dg, CONST_P));
        GFF_TRY(cudaEventRecord(ev[1], h->stream));
        GFF_TRY(launch_galerkin<double>(h, h->d_P, (const double*)nullptr, h->d_b, pa, ores, h->d_spec));
        GFF_TRY(launch_dot<double>(h->d_b, h->d_b, n, h->d_red, h->d_scal, h->stream));
        GFF_TRY(launch_dot<double>(h->d_P, h->d_P, n, h->d_red + RED_BLOCKS, h->d_scal + 1, h->stream));
        GFF_TRY(cudaMemcpyAsync(h->d_scal + 2, h->d_flag, sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
        GFF_TRY(cudaMemcpyAsync(h->d_scal + 3, h->d_flag + 2, sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
        GFF_TRY(cudaMemcpyAsync(h->d_scal + 4, h->d_flag + 4, 2 * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
        GFF_TRY(cudaEventRecord(ev[2], h->stream));
        double s3[5];
        gff_status st2 = fetch(h, h->d_scal, 5, s3);
        if (st2 != GFF_OK) return st2;
        float ms01 = 0.f, ms12 = 0.f;
        GFF_TRY(cudaEventElapsedTime(&ms01, ev[0], ev[1]));
        GFF_TRY(cudaEventElapsedTime(&ms12, ev[1], ev[2]));
        t_const += 1e-3 * ms01;
        t_res += 1e-3 * ms12;
        int flag, tmo, stats[2];
        std::memcpy(&flag, &s3[2], sizeof(int));
        std::memcpy(&tmo, &s3[3], sizeof(int));
        std::memcpy(stats, &s3[4], 2 * sizeof(int));
        cp_fb += stats[0];
        cp_its += (double)stats[1] / (double)N;
        if (tmo) return fail(h, GFF_ERR_TIMEOUT, "a bulk-copy wait in an FFT pass timed out");
        if (flag) return fail(h, GFF_ERR_CP_FAIL, "return map failed in %d voxels", flag);
        rr_b = s3[0];
        nb = std::sqrt(s3[0]);
        nP = std::sqrt(s3[1]);
        res = nP > 0 ? nb / nP : nb;
        return GFF_OK;
    };

    const bool dg_prev = first_eval_warm(h, d9);
    // warm starts: mode 1 keeps the network's guess only if its residual beats the zero
    // start's, mode 2 always, mode 3 extrapolates the last increment without a network
    int wmode = h->opt.warm_start;
    if ((wmode == GFF_WARM_NET_IF_BETTER || wmode == GFF_WARM_NET) && !h->unet) wmode = GFF_WARM_OFF;
    if (wmode) {
        double res_zero = -1.0;
        if (wmode == GFF_WARM_NET_IF_BETTER) {
            if ((st = evaluate(dg_prev)) != GFF_OK) return st;
            res_zero = res;
        }
        int applied = 0;
        cudaError_t e = warm_guess(wmode == GFF_WARM_EXTRAPOLATE ? nullptr : h->unet, h, d9, &applied);
        if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "warm start: %s", cudaGetErrorString(e));
        st = applied ? evaluate(dg_prev) : GFF_OK;
        if (st != GFF_OK && st != GFF_ERR_CP_FAIL) return st;
        warm_used = applied;
        // a guess the return map cannot take, or one with a non-finite residual, is dropped in
        // every mode; mode 1 also drops a guess that does not beat the zero start
        if (!applied) {
            if (wmode != GFF_WARM_NET_IF_BETTER && (st = evaluate(dg_prev)) != GFF_OK) return st;
        } else if (st == GFF_ERR_CP_FAIL || !std::isfinite(res) ||
                   (wmode == GFF_WARM_NET_IF_BETTER && !(res < res_zero))) {
            h->err.clear();
            GFF_TRY(launch_add_const9(h->d_Fk, h->d_F, d9, N, h->stream));
            if ((st = evaluate(dg_prev)) != GFF_OK) return st;
            warm_used = 0;
        }
    } else {
        if ((st = evaluate(dg_prev)) != GFF_OK) return st;
    }
    res_first = res;
    for (int it = 0; it <= h->opt.newton_max; ++it) {
        if (it > 0 && (st = evaluate(true)) != GFF_OK) return st;
        if (res <= h->opt.newton_tol) {
            conv = true;
            break;
        }
        if (it == h->opt.newton_max) break;
        // the tangent only now that a Newton correction needs it (the converged iterate never does)
        {
            GFF_TRY(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
            GFF_TRY(cudaEventRecord(ev[0], h->stream));
            GFF_TRY(launch_constitutive(h, h->d_Fk, dt, mixed ? TANGENT_F32 : TANGENT_F64, false, CONST_K));
            GFF_TRY(cudaEventRecord(ev[1], h->stream));
            int kflag = 0;
            GFF_TRY(cudaMemcpyAsync(&kflag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            GFF_TRY(cudaStreamSynchronize(h->stream));
            float ms01 = 0.f;
            GFF_TRY(cudaEventElapsedTime(&ms01, ev[0], ev[1]));
            t_const += 1e-3 * ms01;
            t_tan += 1e-3 * ms01;
            if (kflag) return fail(h, GFF_ERR_CP_FAIL, "tangent failed in %d voxels", kflag);
        }
        const double stop = std::fmax(h->opt.cg_tol * nb, 0.1 * h->opt.newton_tol * nP);
        int its = 0;
        GFF_TRY(cudaEventRecord(ev[2], h->stream));
        if (!mixed) {
            GFF_TRY(cudaMemcpyAsync(h->d_r, h->d_b, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
            if ((st = cg_solve<double>(h, pa, h->d_x, h->d_r, h->d_p, h->d_Ap, h->d_K, rr_b, stop, &its)) != GFF_OK)
                return st;
            GFF_TRY(launch_axpy_to64<double>(h->d_Fk, h->d_x, n, h->stream));
        } else {
            GFF_TRY(launch_cast64to32(h->d_r32, h->d_b, n, h->stream));
            GFF_TRY(launch_dot<float>(h->d_r32, h->d_r32, n, h->d_red, h->d_scal, h->stream));
            double rr32;
            if ((st = fetch(h, h->d_scal, 1, &rr32)) != GFF_OK) return st;
            if ((st = cg_solve<float>(h, pa, h->d_x32, h->d_r32, h->d_p32, h->d_Ap32, h->d_K32, rr32, stop, &its)) !=
                GFF_OK)
                return st;
            GFF_TRY(launch_axpy_to64<float>(h->d_Fk, h->d_x32, n, h->stream));
        }
        GFF_TRY(cudaEventRecord(ev[3], h->stream));
        GFF_TRY(cudaEventSynchronize(ev[3]));
        float ms23 = 0.f;
        GFF_TRY(cudaEventElapsedTime(&ms23, ev[2], ev[3]));
        t_lin += 1e-3 * ms23;
        cgsum += its;
        ++newton;
    }
    if (!conv) return fail(h, GFF_ERR_NO_CONVERGENCE, "Newton: residual %.3e after %d iterations", res, newton);
    return GFF_OK;
}

}  // namespace

namespace gff {
bool first_eval_warm(const gff_handle* h, const double* d9) {
    if (h->nhist < 1) return false;
    double dd = 0.0, a2 = 0.0, b2 = 0.0;
    for (int c = 0; c < 9; ++c) {
        dd += d9[c] * h->prev_d9[c];
        a2 += d9[c] * d9[c];
        b2 += h->prev_d9[c] * h->prev_d9[c];
    }
    return a2 > 0 && b2 > 0 && dd > 0.5 * std::sqrt(a2 * b2);
}

gff_status record_history(gff_handle* h, const double* d9, const double* dF, cudaStream_t st) {
    double dn = 0.0;
    for (int c = 0; c < 9; ++c) dn += d9[c] * d9[c];
    dn = std::sqrt(dn);
    if (dn > 0) {
        const int slot = h->ycur ^ 1;
        const long long N = h->N;
        GFF_TRY(launch_fluct_incr(h->d_yhist + (size_t)slot * 9 * N, h->d_Fk, h->d_F, dF, 1.0 / dn, N, st));
        h->ycur = slot;
        h->nhist = h->nhist < 2 ? h->nhist + 1 : 2;
    } else {
        h->nhist = 0;  // a purely stress-controlled increment has no direction: history restarts
    }
    for (int c = 0; c < 9; ++c) {
        h->prev2_d9[c] = h->prev_d9[c];
        h->prev_d9[c] = d9[c];
    }
    return GFF_OK;
}

// Grain tables uploaded and launch shapes tuned: what gff_step does before its first increment.
gff_status prepare_for_increments(gff_handle* h) {
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    if (!h->tuned) {
        cudaError_t e = autotune_galerkin(h);
        if (e == cudaSuccess) e = preload_constitutive();
        if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    return GFF_OK;
}
void set_error(gff_handle* h, const char* msg) { h->err = msg; }
}  // namespace gff

namespace {

// Commit the converged iterate: F, internal variables, FIP accumulators, and
// the increment history the warm starts use.
gff_status commit_increment(gff_handle* h, gff_step_report* rep) {
    const long long N = h->N;
    gff_status st;
    double s[27];
    GFF_TRY(launch_sum9(h->d_P, N, h->d_red, h->d_scal, h->stream));
    GFF_TRY(launch_sum9(h->d_Fk, N, h->d_red + 9 * RED_BLOCKS, h->d_scal + 9, h->stream));
    GFF_TRY(launch_sum9(h->d_F, N, h->d_red + 18 * RED_BLOCKS, h->d_scal + 18, h->stream));
    if ((st = fetch(h, h->d_scal, 27, s)) != GFF_OK) return st;
    double dF[9];
    for (int c = 0; c < 9; ++c) {
        rep->Pmacro[c] = s[c] / (double)N;
        rep->Fmacro[c] = s[9 + c] / (double)N;
        dF[c] = (s[9 + c] - s[18 + c]) / (double)N;
    }
    if ((st = record_history(h, h->cur_d9, dF, h->stream)) != GFF_OK) return st;
    GFF_TRY(cudaMemcpyAsync(h->d_F, h->d_Fk, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (h->any_cp) {
        GFF_TRY(cudaMemcpyAsync(h->d_Fpi, h->d_Fpi_t, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        GFF_TRY(cudaMemcpyAsync(h->d_chi, h->d_chi_t, 12 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        GFF_TRY(launch_fip_accumulate(h));
    }
    // the converged iterate's tangent is never computed: K is stale until gff_constitutive
    h->K_valid = h->K32_valid = false;
    for (int c = 0; c < 9; ++c) h->Pmacro_committed[c] = rep->Pmacro[c];
    GFF_TRY(cudaStreamSynchronize(h->stream));
    return GFF_OK;
}

// One increment; when Newton or a return map fails, the increment is split
// into two halves (dt/2; macroscopic F and P interpolated from the last
// committed state) and retried, down to max_cuts levels.  Nothing is
// committed by a failed attempt, so each retry starts from the same state.
gff_status step_with_cuts(gff_handle* h, double dt, const double* Fbar, const uint8_t* mask, const double* Pbar,
                          int depth, gff_step_report* acc) {
    gff_step_report rep;
    std::memset(&rep, 0, sizeof rep);
    gff_status st = newton_increment(h, dt, Fbar, mask, Pbar, &rep);
    acc->newton_iters += rep.newton_iters;
    acc->cg_iters += rep.cg_iters;
    acc->t_constitutive += rep.t_constitutive;
    acc->t_residual += rep.t_residual;
    acc->t_linear += rep.t_linear;
    acc->cp_fallbacks += rep.cp_fallbacks;
    acc->cp_local_iters += rep.cp_local_iters;
    acc->t_tangent += rep.t_tangent;
    acc->residual = rep.residual;
    if (depth == 0) {
        acc->warm_start_used = rep.warm_start_used;
        acc->residual_first = rep.residual_first;
    }
    if (st == GFF_OK) return commit_increment(h, acc);
    if ((st != GFF_ERR_CP_FAIL && st != GFF_ERR_NO_CONVERGENCE) || depth >= h->opt.max_cuts) return st;
    // macroscopic state of the last commit
    double Fsum[9];
    GFF_TRY(launch_sum9(h->d_F, h->N, h->d_red, h->d_scal, h->stream));
    if ((st = fetch(h, h->d_scal, 9, Fsum)) != GFF_OK) return st;
    double Fmid[9], Pmid[9];
    for (int c = 0; c < 9; ++c) {
        Fmid[c] = 0.5 * (Fsum[c] / (double)h->N + Fbar[c]);
        Pmid[c] = 0.5 * (h->Pmacro_committed[c] + Pbar[c]);
    }
    ++acc->cuts;
    h->err.clear();
    if ((st = step_with_cuts(h, 0.5 * dt, Fmid, mask, Pmid, depth + 1, acc)) != GFF_OK) return st;
    return step_with_cuts(h, 0.5 * dt, Fbar, mask, Pbar, depth + 1, acc);
}

}  // namespace

GFF_EXPORT gff_status gff_step(gff_handle* h, double dt, const double Fbar[9], const uint8_t mask[9], const double Pbar[9],
                    gff_step_report* report) {
    if (!h || !Fbar || !mask || !Pbar || !(dt > 0)) return fail(h, GFF_ERR_ARG, "bad step args");
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    gff_step_report rep;
    std::memset(&rep, 0, sizeof rep);
    if (!h->tuned) {
        GFF_TRY(autotune_galerkin(h));
        GFF_TRY(preload_constitutive());
    }
    st = step_with_cuts(h, dt, Fbar, mask, Pbar, 0, &rep);
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (report) *report = rep;
    return st;
}

GFF_EXPORT gff_status gff_run_history(gff_handle* h, int nsteps, const double* dt, const double* Fbar, const uint8_t* mask,
                           const double* Pbar, const uint8_t* cycle_start, double* Pmacro_out,
                           gff_step_report* reports) {
    if (!h || nsteps < 0 || !dt || !Fbar || !mask || !Pbar) return fail(h, GFF_ERR_ARG, "bad history args");
    for (int k = 0; k < nsteps; ++k) {
        if (cycle_start && cycle_start[k]) {
            gff_status st = gff_reset_fips(h);
            if (st != GFF_OK) return st;
        }
        gff_step_report rep;
        gff_status st = gff_step(h, dt[k], Fbar + 9 * k, mask + 9 * k, Pbar + 9 * k, &rep);
        if (reports) reports[k] = rep;
        if (st != GFF_OK) return st;
        if (Pmacro_out) std::memcpy(Pmacro_out + 9 * k, rep.Pmacro, 9 * sizeof(double));
    }
    return GFF_OK;
}

GFF_EXPORT void gff_auto_options_default(gff_auto_options* a) {
    if (!a) return;
    a->dt_initial = 0.05;
    a->dt_min = 1e-6;
    a->dt_max = 1.0;
    a->grow = 1.5;
    a->shrink = 0.75;
    a->easy_newton = 3;
    a->hard_newton = 8;
}

// Automatic time incrementation along a piecewise-linear macroscopic path.
GFF_EXPORT gff_status gff_run_auto(gff_handle* h, int nknots, const double* t_knots, const double* Fbar_knots,
                                   const uint8_t* mask, const double* Pbar_knots, const uint8_t* cycle_start,
                                   const gff_auto_options* ao, int max_increments, int* n_out, double* t_out,
                                   double* Pmacro_out, gff_step_report* reports) {
    if (!h || nknots < 2 || !t_knots || !Fbar_knots || !mask || !Pbar_knots || !ao || max_increments < 1 || !n_out)
        return fail(h, GFF_ERR_ARG, "bad automatic-incrementation args");
    for (int k = 1; k < nknots; ++k)
        if (!(t_knots[k] > t_knots[k - 1])) return fail(h, GFF_ERR_ARG, "knot times must increase");
    if (!(ao->dt_min > 0) || !(ao->dt_initial >= ao->dt_min) || !(ao->dt_max >= ao->dt_initial) || !(ao->grow >= 1) ||
        !(ao->shrink > 0 && ao->shrink <= 1) || ao->easy_newton < 0 || ao->hard_newton <= ao->easy_newton)
        return fail(h, GFF_ERR_ARG, "automatic-incrementation options out of range");
    *n_out = 0;
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    double t = t_knots[0], dt = ao->dt_initial;
    int seg = 0;  // current knot interval [t_knots[seg], t_knots[seg + 1]]
    const double tend = t_knots[nknots - 1];
    const double eps_t = 1e-12 * (tend - t_knots[0]);
    while (t < tend - eps_t) {
        if (*n_out >= max_increments) return fail(h, GFF_ERR_NO_CONVERGENCE, "more than %d increments needed", max_increments);
        while (seg + 1 < nknots - 1 && t >= t_knots[seg + 1] - eps_t) ++seg;
        // a knot flagged as a cycle start restarts the FIP accumulators when the path reaches it
        if (cycle_start && std::fabs(t - t_knots[seg]) <= eps_t && cycle_start[seg]) {
            if ((st = gff_reset_fips(h)) != GFF_OK) return st;
        }
        double t1 = t + dt;
        if (t1 > t_knots[seg + 1] - eps_t) t1 = t_knots[seg + 1];  // never step across a knot
        const double w = (t1 - t_knots[seg]) / (t_knots[seg + 1] - t_knots[seg]);
        double Fb[9], Pb[9];
        for (int c = 0; c < 9; ++c) {
            Fb[c] = (1 - w) * Fbar_knots[9 * seg + c] + w * Fbar_knots[9 * (seg + 1) + c];
            Pb[c] = (1 - w) * Pbar_knots[9 * seg + c] + w * Pbar_knots[9 * (seg + 1) + c];
        }
        gff_step_report rep;
        st = gff_step(h, t1 - t, Fb, mask, Pb, &rep);
        if (reports) reports[*n_out] = rep;
        if (st != GFF_OK) return st;
        if (t_out) t_out[*n_out] = t1;
        if (Pmacro_out) std::memcpy(Pmacro_out + 9 * *n_out, rep.Pmacro, 9 * sizeof(double));
        ++*n_out;
        const double taken = t1 - t;
        t = t1;
        // the next step: the size that worked after cut-backs, grown after an easy
        // increment, shrunk after a hard one; within [dt_min, dt_max]
        double nd = dt;
        if (rep.cuts > 0)
            nd = taken * std::ldexp(1.0, -rep.cuts);
        else if (rep.newton_iters <= ao->easy_newton && taken >= 0.999 * dt)
            nd = dt * ao->grow;
        else if (rep.newton_iters >= ao->hard_newton)
            nd = dt * ao->shrink;
        dt = std::min(std::max(nd, ao->dt_min), ao->dt_max);
    }
    return GFF_OK;
}

GFF_EXPORT gff_status gff_reset_fips(gff_handle* h) {
    if (!h) return GFF_ERR_ARG;
    GFF_TRY(launch_fip_reset(h));
    GFF_TRY(cudaStreamSynchronize(h->stream));
    return GFF_OK;
}

GFF_EXPORT gff_status gff_get_fips(gff_handle* h, double* pcyc_g, double* wcyc_g, double* fs_g) {
    if (!h) return GFF_ERR_ARG;
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    const int ng = h->ngrains;
    double* d = nullptr;
    if ((st = dalloc(h, (void**)&d, (14 + 38) * (size_t)ng * sizeof(double), "grain fips")) != GFF_OK) return st;
    cudaError_t e = launch_grain_fips(h, d, d + ng, d + 13 * (size_t)ng);
    std::vector<double> host(14 * (size_t)ng);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), d, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "grain fips: %s", cudaGetErrorString(e));
    if (pcyc_g) std::memcpy(pcyc_g, host.data(), ng * sizeof(double));
    if (wcyc_g) std::memcpy(wcyc_g, host.data() + ng, 12 * (size_t)ng * sizeof(double));
    if (fs_g) std::memcpy(fs_g, host.data() + 13 * (size_t)ng, ng * sizeof(double));
    return GFF_OK;
}

GFF_EXPORT gff_status gff_umat_tangent(long long n, const double* F_dev, const double* sigma_dev, const double* Cab_dev,
                                       double* P_dev, double* K_dev, void* stream) {
    if (n < 0 || (n > 0 && (!F_dev || !sigma_dev || !Cab_dev || !P_dev || !K_dev))) return GFF_ERR_ARG;
    if (n == 0) return GFF_OK;
    cudaError_t e = launch_umat_convert(n, F_dev, sigma_dev, Cab_dev, P_dev, K_dev, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GFF_OK : GFF_ERR_CUDA;
}

GFF_EXPORT gff_status gff_get_band_fips(gff_handle* h, double width, double* wb_g, double* wb_max) {
    if (!h || !(width > 0)) return fail(h, GFF_ERR_ARG, "band width must be positive");
    gff_status st = ensure_grains(h);
    if (st != GFF_OK) return st;
    const int ng = h->ngrains;
    const double smax = 0.5 * std::sqrt(h->grid.L[0] * h->grid.L[0] + h->grid.L[1] * h->grid.L[1] +
                                        h->grid.L[2] * h->grid.L[2]);
    const double nbd = 2.0 * (std::floor(smax / width) + 2.0);
    if (nbd * ng * 16.0 * sizeof(double) > 2e9)
        return fail(h, GFF_ERR_ARG, "band width %.3e too small for %d grains (more than 2 GB of band sums)", width, ng);
    const int NB = (int)nbd;
    void* scratch = nullptr;
    const size_t bytes = band_scratch_bytes(ng, NB) + (size_t)ng * sizeof(double);
    if ((st = dalloc(h, &scratch, bytes, "band sums")) != GFF_OK) return st;
    double* out = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + band_scratch_bytes(ng, NB));
    std::vector<double> host(ng);
    cudaError_t e = launch_band_fips(h, width, NB, scratch, out);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), out, ng * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(h, GFF_ERR_CUDA, "band fips: %s", cudaGetErrorString(e));
    if (wb_g) std::memcpy(wb_g, host.data(), ng * sizeof(double));
    if (wb_max) *wb_max = *std::max_element(host.begin(), host.end());
    return GFF_OK;
}

// ------------------------------------------------------------------ checkpoint
static const char kMagic[8] = {'G', 'F', 'F', 'S', 'T', 'A', 'T', '2'};

// Host part of the increment history: everything the next increment's start reads.
struct HistHeader {
    int32_t nhist, ycur, pad[2];
    double prev_d9[9], prev2_d9[9], Pmacro[9];
};

GFF_EXPORT gff_status gff_save_state(gff_handle* h, const char* path) {
    if (!h || !path) return fail(h, GFF_ERR_ARG, "bad args");
    const long long N = h->N;
    const size_t counts[5] = {9 * (size_t)N, 9 * (size_t)N, 12 * (size_t)N, NACC * (size_t)N, 12 * (size_t)N};
    double* src[5] = {h->d_F, h->d_Fpi, h->d_chi, h->d_acc, h->d_dg};
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, GFF_ERR_IO, "cannot open %s", path);
    int32_t hdr[4] = {h->grid.nx, h->grid.ny, h->grid.nz, NACC};
    HistHeader hh{};
    hh.nhist = h->nhist;
    hh.ycur = h->ycur;
    for (int c = 0; c < 9; ++c) {
        hh.prev_d9[c] = h->prev_d9[c];
        hh.prev2_d9[c] = h->prev2_d9[c];
        hh.Pmacro[c] = h->Pmacro_committed[c];
    }
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(&hh, sizeof hh, 1, f) == 1;
    std::vector<double> buf;
    for (int i = 0; i < 5 && ok; ++i) {
        buf.resize(counts[i]);
        cudaError_t e = cudaMemcpy(buf.data(), src[i], counts[i] * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(h, GFF_ERR_CUDA, "save: %s", cudaGetErrorString(e));
        }
        ok = std::fwrite(buf.data(), sizeof(double), counts[i], f) == counts[i];
    }
    if (ok) {
        std::vector<float> yb(18 * (size_t)N);
        cudaError_t e = cudaMemcpy(yb.data(), h->d_yhist, yb.size() * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(h, GFF_ERR_CUDA, "save: %s", cudaGetErrorString(e));
        }
        ok = std::fwrite(yb.data(), sizeof(float), yb.size(), f) == yb.size();
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? GFF_OK : fail(h, GFF_ERR_IO, "write failed: %s", path);
}

GFF_EXPORT gff_status gff_load_state(gff_handle* h, const char* path) {
    if (!h || !path) return fail(h, GFF_ERR_ARG, "bad args");
    const long long N = h->N;
    const size_t counts[5] = {9 * (size_t)N, 9 * (size_t)N, 12 * (size_t)N, NACC * (size_t)N, 12 * (size_t)N};
    double* dst[5] = {h->d_F, h->d_Fpi, h->d_chi, h->d_acc, h->d_dg};
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, GFF_ERR_IO, "cannot open %s", path);
    char mg[8];
    int32_t hdr[4];
    HistHeader hh{};
    bool ok = std::fread(mg, 1, 8, f) == 8 && std::memcmp(mg, kMagic, 8) == 0 && std::fread(hdr, sizeof hdr, 1, f) == 1;
    if (ok && (hdr[0] != h->grid.nx || hdr[1] != h->grid.ny || hdr[2] != h->grid.nz || hdr[3] != NACC)) {
        std::fclose(f);
        return fail(h, GFF_ERR_ARG, "state file grid %dx%dx%d does not match", hdr[0], hdr[1], hdr[2]);
    }
    ok = ok && std::fread(&hh, sizeof hh, 1, f) == 1 && hh.nhist >= 0 && hh.nhist <= 2 && (hh.ycur == 0 || hh.ycur == 1);
    std::vector<double> buf;
    for (int i = 0; i < 5 && ok; ++i) {
        buf.resize(counts[i]);
        ok = std::fread(buf.data(), sizeof(double), counts[i], f) == counts[i];
        if (ok) {
            cudaError_t e = cudaMemcpy(dst[i], buf.data(), counts[i] * sizeof(double), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                std::fclose(f);
                return fail(h, GFF_ERR_CUDA, "load: %s", cudaGetErrorString(e));
            }
        }
    }
    if (ok) {
        std::vector<float> yb(18 * (size_t)N);
        ok = std::fread(yb.data(), sizeof(float), yb.size(), f) == yb.size();
        if (ok) {
            cudaError_t e = cudaMemcpy(h->d_yhist, yb.data(), yb.size() * sizeof(float), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                std::fclose(f);
                return fail(h, GFF_ERR_CUDA, "load: %s", cudaGetErrorString(e));
            }
        }
    }
    std::fclose(f);
    if (!ok) return fail(h, GFF_ERR_IO, "read failed or not a state file: %s", path);
    GFF_TRY(cudaMemcpy(h->d_Fk, h->d_F, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice));
    h->K_valid = h->K32_valid = false;
    h->nhist = hh.nhist;
    h->ycur = hh.ycur;
    for (int c = 0; c < 9; ++c) {
        h->prev_d9[c] = hh.prev_d9[c];
        h->prev2_d9[c] = hh.prev2_d9[c];
        h->Pmacro_committed[c] = hh.Pmacro[c];
    }
    return GFF_OK;
}

