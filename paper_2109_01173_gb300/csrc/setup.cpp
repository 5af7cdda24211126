// Host-side setup of libmofem: 1D FEM factors, boundary trimming, the operator's
// term tables, the RHS mass factors and the preconditioner pencils with their
// generalized eigendecompositions (FP64, cuSOLVER on the GPU).
//
// Paper sections: Sec. 2.2 (map eta and H^), Sec. 3.1-3.3 (1D stiffness, mass
// and weighted matrices, Eqs. stiffness_mass_1D and newmatrix_1..7; lumped P1 via
// the element-wise interpolant I_h), the Dirichlet remark (trimming, Eq.
// variable_dimension), Sec. 4 (reduced approach, Eq. diagonalisation_1).
//
// Two-profile generalisation: domain {0<=x<=1, g1(x)<=y<=g2(x)}, map
// (s,t) -> (s, g1(s) + t h(s)), h = g2 - g1, w = g1' + t h'.  The pulled-back
// bilinear form splits into eight Kronecker terms S (x) T acting as U -> S U T^T:
//   (K_s[h] + gamma M_s[h]) (x) M_t,   M_s[(1+g1'^2)/h] (x) K_t,
//   M_s[2 g1' h'/h] (x) K_t[t],        M_s[h'^2/h] (x) K_t[t^2],
//   -G_s[g1'] (x) C_t^T, -G_s[g1']^T (x) C_t, -G_s[h'] (x) C_t[t]^T, -G_s[h']^T (x) C_t[t],
// with K[w] = int psi' psi' w, M[w] = int psi psi w, G[w]_ij = int psi_i' psi_j w.
// When g1' vanishes the 3rd, 5th and 6th terms drop and the remaining five
// are the paper's Eq. kronecker_mass_distorted.
#include "internal.h"

#include <cusolverDn.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

static thread_local std::string g_last_error;
void mofem_set_last_error(const char* msg, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s (%s:%d)", msg, file, line);
    g_last_error = buf;
}
extern "C" const char* mofem_last_error() { return g_last_error.c_str(); }

namespace {

// Gauss-Legendre nodes/weights on [0, 1] by Newton's method on P_m with the
// three-term recurrence (m + 1) P_{m+1} = (2m + 1) x P_m - m P_{m-1}.
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= m; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pm = (m == 1) ? z : p1;
            double pm1 = (m == 1) ? 1.0 : p0;
            dp = m * (z * pm - pm1) / (z * z - 1.0);
            double dz = pm / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged root
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= m; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        double pm = (m == 1) ? z : p1, pm1 = (m == 1) ? 1.0 : p0;
        dp = m * (z * pm - pm1) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);   // map [-1,1] -> [0,1]
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // = 2/((1-z^2) P'^2) / 2
    }
}

// Lagrange basis of degree d on nodes j/d and its xi-derivative at point xi.
void lagrange(int d, double xi, double* val, double* der) {
    for (int j = 0; j <= d; ++j) {
        double xj = double(j) / d;
        double v = 1.0, den = 1.0, dv = 0.0;
        for (int m = 0; m <= d; ++m) {
            if (m == j) continue;
            double xm = double(m) / d;
            den *= (xj - xm);
            // d/dxi of running product: (v * (xi - xm))' = dv (xi - xm) + v
            dv = dv * (xi - xm) + v;
            v *= (xi - xm);
        }
        val[j] = v / den;
        der[j] = dv / den;
    }
}

struct Quad {
    int E, d, nq;
    double hE;
    std::vector<double> xi, wq;           // reference rule
    std::vector<double> phi, dphi;        // [nq][d+1]
    std::vector<double> x;                // physical points [E][nq]
};

Quad make_quad(int n, int k, int nq_opt) {
    Quad Qd;
    Qd.d = (k == 0) ? 1 : k;
    Qd.E = (n - 1) / Qd.d;
    Qd.hE = 1.0 / Qd.E;
    if (k == 0) {   // lumped P1: integrate the element-wise linear interpolant (trapezoid)
        Qd.xi = {0.0, 1.0};
        Qd.wq = {0.5, 0.5};
    } else {
        gauss_legendre(nq_opt > 0 ? nq_opt : k + 3, Qd.xi, Qd.wq);
    }
    Qd.nq = (int)Qd.xi.size();
    Qd.phi.resize(Qd.nq * (Qd.d + 1));
    Qd.dphi.resize(Qd.nq * (Qd.d + 1));
    for (int i = 0; i < Qd.nq; ++i) lagrange(Qd.d, Qd.xi[i], &Qd.phi[i * (Qd.d + 1)], &Qd.dphi[i * (Qd.d + 1)]);
    Qd.x.resize(Qd.E * Qd.nq);
    for (int e = 0; e < Qd.E; ++e)
        for (int i = 0; i < Qd.nq; ++i) Qd.x[e * Qd.nq + i] = (e + Qd.xi[i]) * Qd.hE;
    return Qd;
}

// Banded n x n matrix, band[r*P + j] = A[r][r + j - K].
struct Band {
    int n = 0, K = 0, P = 0;
    std::vector<double> v;
    Band() {}
    Band(int n_, int K_) : n(n_), K(K_), P(2 * K_ + 1), v((size_t)n_ * (2 * K_ + 1), 0.0) {}
    double& at(int r, int c) { return v[(size_t)r * P + (c - r + K)]; }
    double get(int r, int c) const {
        if (r < 0 || r >= n || c < 0 || c >= n || c - r < -K || c - r > K) return 0.0;
        return v[(size_t)r * P + (c - r + K)];
    }
};

enum Kind { KIND_K, KIND_M, KIND_G };

// Weighted 1D matrix: K[w], M[w] or G[w], weight given at the quadrature points.
Band assemble(const Quad& Qd, int n, Kind kind, const std::vector<double>& w) {
    const int d = Qd.d;
    Band A(n, d);
    for (int e = 0; e < Qd.E; ++e) {
        for (int iq = 0; iq < Qd.nq; ++iq) {
            const double* ph = &Qd.phi[iq * (d + 1)];
            const double* dp = &Qd.dphi[iq * (d + 1)];
            double ww = Qd.wq[iq] * Qd.hE * w[e * Qd.nq + iq];
            for (int a = 0; a <= d; ++a) {
                double la = (kind == KIND_M) ? ph[a] : dp[a] / Qd.hE;
                for (int c = 0; c <= d; ++c) {
                    double rc = (kind == KIND_K) ? dp[c] / Qd.hE : ph[c];
                    A.at(e * d + a, e * d + c) += ww * la * rc;
                }
            }
        }
    }
    return A;
}

Band add(const Band& A, const Band& B, double sb) {
    Band C = A;
    for (size_t i = 0; i < C.v.size(); ++i) C.v[i] += sb * B.v[i];
    return C;
}

// Trimmed diagonal-major table: out[j*q + r] = A[r+off][r+off+j-K] if the column
// is kept, for kept rows r = 0..q-1.  transpose -> use A^T; scale multiplies.
void trimmed_table(const Band& A, int q, int off, int col_lo, int col_hi, bool transpose, double scale,
                   double* out) {
    const int K = A.K, P = A.P;
    for (int j = 0; j < P; ++j)
        for (int r = 0; r < q; ++r) {
            int row = r + off, col = row + j - K;
            double v = 0.0;
            if (col >= col_lo && col <= col_hi) v = transpose ? A.get(col, row) : A.get(row, col);
            out[(size_t)j * q + r] = scale * v;
        }
}

void dense_trimmed(const Band& A, int q, int off, std::vector<double>& D) {
    D.assign((size_t)q * q, 0.0);
    for (int r = 0; r < q; ++r)
        for (int c = r - A.K; c <= r + A.K; ++c)
            if (c >= 0 && c < q) D[(size_t)r * q + c] = A.get(r + off, c + off);
}

template <class T>
mofem_status dev_alloc(T** p, size_t count) {
    MOFEM_CUDA_TRY(cudaMalloc((void**)p, count * sizeof(T)));
    return MOFEM_OK;
}

}  // namespace

// Everything the setup computes on the host, before any device work.
struct HostTables {
    int NT = 5, K = 1, P = 3, q = 0, off = 1, nq = 0;
    std::vector<double> S, T, Srh, Trh;   // [B][NT][P][q], [NT][P][q], [B][P][q], [P][q]
    std::vector<double> Smf, Tmf;         // untrimmed masses M_s[h], M_t: [B][P][n], [P][n]
    std::vector<Band> E1s, E2s;
    Band Mt, Kt;
    Band F1, F2;                          // t-pencil F2 Q2 = F1 Q2 diag(mu)
};

// Identity as a band of half-width K.
static Band identity_band(int n, int K) {
    Band I(n, K);
    for (int r = 0; r < n; ++r) I.at(r, r) = 1.0;
    return I;
}

static mofem_status build_host_tables(int B, int k, int n, mofem_bc bc, const mofem_opts& opts,
                                      const mofem_profile* g1, const mofem_profile* g2, const double* gamma,
                                      HostTables& H);

static mofem_status build_host_tables(int B, int k, int n, mofem_bc bc, const mofem_opts& opts,
                                      const mofem_profile* g1, const mofem_profile* g2, const double* gamma,
                                      HostTables& H) {
    Quad Qd = make_quad(n, k, opts.quad_points);
    H.K = Qd.d;
    H.P = 2 * H.K + 1;
    H.nq = Qd.nq;
    H.off = (bc == MOFEM_BC_DIRICHLET) ? 1 : 0;
    H.q = (bc == MOFEM_BC_DIRICHLET) ? n - 2 : n;
    const int q = H.q, P = H.P, off = H.off;
    const int lo = off, hi = n - 1 - off;   // kept node range
    const int nqt = Qd.E * Qd.nq;

    // --- per-instance geometry at the quadrature points ---------------------
    std::vector<std::vector<double>> wh(B), wa(B), wb(B), wc(B), wg1(B), wdh(B), we2(B);
    bool any_g1 = false;
    for (int i = 0; i < B; ++i) {
        wh[i].resize(nqt); wa[i].resize(nqt); wb[i].resize(nqt); wc[i].resize(nqt);
        wg1[i].resize(nqt); wdh[i].resize(nqt); we2[i].resize(nqt);
        for (int p = 0; p < nqt; ++p) {
            double s = Qd.x[p];
            double a1 = g1[i].g(s, g1[i].ctx), a2 = g2[i].g(s, g2[i].ctx);
            double d1 = g1[i].dg(s, g1[i].ctx), d2 = g2[i].dg(s, g2[i].ctx);
            double h = a2 - a1, dh = d2 - d1;
            if (!(h > 0.0) || !std::isfinite(h) || !std::isfinite(dh) || !std::isfinite(d1)) {
                mofem_set_last_error("profile: h = g2 - g1 must be positive and finite", __FILE__, __LINE__);
                return MOFEM_ERR_INVALID_ARG;
            }
            wh[i][p] = h;
            wa[i][p] = (1.0 + d1 * d1) / h;
            wb[i][p] = 2.0 * d1 * dh / h;
            wc[i][p] = dh * dh / h;
            wg1[i][p] = d1;
            wdh[i][p] = dh;
            // t-average over [0,1] of (1 + (g1' + t h')^2)/h
            we2[i][p] = (opts.pencil == MOFEM_PENCIL_DOMINANT)
                            ? wa[i][p]
                            : (1.0 + d1 * d1 + d1 * dh + dh * dh / 3.0) / h;
            if (d1 != 0.0) any_g1 = true;
        }
    }
    H.NT = any_g1 ? 8 : 5;
    const int NT = H.NT;

    // --- t-direction factors (shared) ---------------------------------------
    std::vector<double> ones(nqt, 1.0), tw(nqt), tw2(nqt);
    for (int p = 0; p < nqt; ++p) { tw[p] = Qd.x[p]; tw2[p] = Qd.x[p] * Qd.x[p]; }
    Band Mt = assemble(Qd, n, KIND_M, ones);
    Band Kt = assemble(Qd, n, KIND_K, ones);
    Band Ktt = assemble(Qd, n, KIND_K, tw);
    Band Ktt2 = assemble(Qd, n, KIND_K, tw2);
    Band Ct1 = assemble(Qd, n, KIND_G, ones);
    Band Ctt = assemble(Qd, n, KIND_G, tw);
    H.Mt = Mt;
    H.Kt = Kt;
    // t-pencil F2 Q2 = F1 Q2 diag(mu).  Single-term preconditioners E Z F^T take the
    // standard eigenpairs of F (F1 = I): PRODUCT F = K_t + K_t[t^2]; PARABOLIC F = M_t +
    // (K_t + K_t[t^2]) / gamma (the IMEX step scaled by 1/(d_u tau)); AUA F = K_t.
    const bool single = opts.pencil == MOFEM_PENCIL_PRODUCT || opts.pencil == MOFEM_PENCIL_PARABOLIC ||
                        opts.pencil == MOFEM_PENCIL_AUA;
    H.F1 = single ? identity_band(n, Mt.K) : Mt;
    if (opts.pencil == MOFEM_PENCIL_PRODUCT) H.F2 = add(Kt, Ktt2, 1.0);
    else if (opts.pencil == MOFEM_PENCIL_PARABOLIC) H.F2 = add(Mt, add(Kt, Ktt2, 1.0), 1.0 / gamma[0]);
    else H.F2 = Kt;

    std::vector<double>& Th = H.T;
    Th.assign((size_t)NT * P * q, 0.0);
    auto tslot = [&](int i) { return Th.data() + (size_t)i * P * q; };
    if (NT == 5) {
        trimmed_table(Mt, q, off, lo, hi, false, 1.0, tslot(0));
        trimmed_table(Kt, q, off, lo, hi, false, 1.0, tslot(1));
        trimmed_table(Ktt2, q, off, lo, hi, false, 1.0, tslot(2));
        trimmed_table(Ctt, q, off, lo, hi, true, 1.0, tslot(3));
        trimmed_table(Ctt, q, off, lo, hi, false, 1.0, tslot(4));
    } else {
        trimmed_table(Mt, q, off, lo, hi, false, 1.0, tslot(0));
        trimmed_table(Kt, q, off, lo, hi, false, 1.0, tslot(1));
        trimmed_table(Ktt, q, off, lo, hi, false, 1.0, tslot(2));
        trimmed_table(Ktt2, q, off, lo, hi, false, 1.0, tslot(3));
        trimmed_table(Ct1, q, off, lo, hi, true, 1.0, tslot(4));
        trimmed_table(Ct1, q, off, lo, hi, false, 1.0, tslot(5));
        trimmed_table(Ctt, q, off, lo, hi, true, 1.0, tslot(6));
        trimmed_table(Ctt, q, off, lo, hi, false, 1.0, tslot(7));
    }
    // RHS t-factor: rows = kept nodes, columns = all nodes
    H.Trh.assign((size_t)P * q, 0.0);
    trimmed_table(Mt, q, off, 0, n - 1, false, 1.0, H.Trh.data());
    // untrimmed t-mass (rows and columns = all nodes): transpose of the right-hand side's map
    H.Tmf.assign((size_t)P * n, 0.0);
    trimmed_table(Mt, n, 0, 0, n - 1, false, 1.0, H.Tmf.data());

    // --- s-direction factors per instance ------------------------------------
    std::vector<double>& Sh = H.S;
    Sh.assign((size_t)B * NT * P * q, 0.0);
    H.Srh.assign((size_t)B * P * q, 0.0);
    H.Smf.assign((size_t)B * P * n, 0.0);
    H.E1s.resize(B);
    H.E2s.resize(B);
    for (int i = 0; i < B; ++i) {
        Band Ksh = assemble(Qd, n, KIND_K, wh[i]);
        Band Msh = assemble(Qd, n, KIND_M, wh[i]);
        Band Msa = assemble(Qd, n, KIND_M, wa[i]);
        Band Msc = assemble(Qd, n, KIND_M, wc[i]);
        Band Gdh = assemble(Qd, n, KIND_G, wdh[i]);
        Band S0 = add(Ksh, Msh, gamma[i]);
        double* base = Sh.data() + (size_t)i * NT * P * q;
        auto sslot = [&](int t) { return base + (size_t)t * P * q; };
        if (NT == 5) {
            trimmed_table(S0, q, off, lo, hi, false, 1.0, sslot(0));
            trimmed_table(Msa, q, off, lo, hi, false, 1.0, sslot(1));
            trimmed_table(Msc, q, off, lo, hi, false, 1.0, sslot(2));
            trimmed_table(Gdh, q, off, lo, hi, false, -1.0, sslot(3));
            trimmed_table(Gdh, q, off, lo, hi, true, -1.0, sslot(4));
        } else {
            Band Msb = assemble(Qd, n, KIND_M, wb[i]);
            Band Gg1 = assemble(Qd, n, KIND_G, wg1[i]);
            trimmed_table(S0, q, off, lo, hi, false, 1.0, sslot(0));
            trimmed_table(Msa, q, off, lo, hi, false, 1.0, sslot(1));
            trimmed_table(Msb, q, off, lo, hi, false, 1.0, sslot(2));
            trimmed_table(Msc, q, off, lo, hi, false, 1.0, sslot(3));
            trimmed_table(Gg1, q, off, lo, hi, false, -1.0, sslot(4));
            trimmed_table(Gg1, q, off, lo, hi, true, -1.0, sslot(5));
            trimmed_table(Gdh, q, off, lo, hi, false, -1.0, sslot(6));
            trimmed_table(Gdh, q, off, lo, hi, true, -1.0, sslot(7));
        }
        trimmed_table(Msh, q, off, 0, n - 1, false, 1.0, H.Srh.data() + (size_t)i * P * q);
        trimmed_table(Msh, n, 0, 0, n - 1, false, 1.0, H.Smf.data() + (size_t)i * P * n);
        if (opts.pencil == MOFEM_PENCIL_PRODUCT || opts.pencil == MOFEM_PENCIL_AUA) {
            // K_s[h] Z F^T: standard eigenpairs on each side
            H.E1s[i] = Ksh;
            H.E2s[i] = identity_band(n, Ksh.K);
        } else if (opts.pencil == MOFEM_PENCIL_PARABOLIC) {   // (K_s[h] + gamma M_s[h]) Z F^T
            H.E1s[i] = S0;
            H.E2s[i] = identity_band(n, S0.K);
        } else {
            H.E1s[i] = S0;
            H.E2s[i] = (opts.pencil == MOFEM_PENCIL_DOMINANT) ? Msa : assemble(Qd, n, KIND_M, we2[i]);
        }
    }
    return MOFEM_OK;
}

// Double-float difference-form tables from the plain FP64 tables S [B][NT][P][q] and
// T [NT][P][q]: each output is a hi plane followed by a lo plane of the same shape.  Off
// the diagonal slot: the coefficient split into (hi, lo).  On it: the exact row sum of
// the FP64 coefficients (TwoSum accumulation, then its (hi, lo) pair) for every t-table
// and for the s-tables of the terms whose s-pass runs in difference form (0, 3, 4 of
// five terms; 0, 4..7 of eight), the plain diagonal coefficient for the others.  Term
// 0's t-table holds N = D^{-1}(M_t - D) off the diagonal and D = rowsum M_t on it (the
// exact mass split of d M_t^T = D (d + d N^T)).  The row sum enters exactly so that,
// with differences of the input taken exactly, no rounding that a stiffness factor
// amplifies is larger than the differences themselves.
static void build_dd_tables(const std::vector<double>& Sh, const std::vector<double>& Th, int B, int NT, int P, int K,
                     int q, std::vector<float>& Sd, std::vector<float>& Td) {
    const unsigned dmask = NT == 5 ? 0x19u : 0xF1u;   // s-passes in difference form
    auto exact_rowsum = [&](const double* base, int r, double& s, double& e) {
        s = 0.0;
        e = 0.0;
        for (int j = 0; j < P; ++j) {
            const double a = base[(size_t)j * q + r];
            const double t = s + a, v = t - s;
            e += (s - (t - v)) + (a - v);
            s = t;
        }
    };
    auto put = [](float* hi, float* lo, size_t i, double s, double e) {
        const float h = (float)s;
        hi[i] = h;
        lo[i] = (float)((s - (double)h) + e);
    };
    Sd.assign(2 * Sh.size(), 0.f);
    Td.assign(2 * Th.size(), 0.f);
    float *sh = Sd.data(), *sl = Sd.data() + Sh.size(), *th = Td.data(), *tl = Td.data() + Th.size();
    for (int t = 0; t < NT; ++t) {
        const double* base = Th.data() + (size_t)t * P * q;
        for (int r = 0; r < q; ++r) {
            double s, e;
            exact_rowsum(base, r, s, e);
            const double d = s + e;
            for (int j = 0; j < P; ++j) {
                const size_t o = (size_t)t * P * q + (size_t)j * q + r;
                if (j == K) put(th, tl, o, s, e);
                else if (t == 0 && NT > 1) put(th, tl, o, d != 0.0 ? base[(size_t)j * q + r] / d : 0.0, 0.0);
                else put(th, tl, o, base[(size_t)j * q + r], 0.0);
            }
        }
    }
    for (int i = 0; i < B; ++i)
        for (int t = 0; t < NT; ++t) {
            const size_t b0 = ((size_t)i * NT + t) * P * q;
            const double* base = Sh.data() + b0;
            const bool diff = (dmask >> t) & 1u;
            for (int r = 0; r < q; ++r) {
                double s = 0.0, e = 0.0;
                if (diff) exact_rowsum(base, r, s, e);
                for (int j = 0; j < P; ++j) {
                    const size_t o = b0 + (size_t)j * q + r;
                    if (diff && j == K) put(sh, sl, o, s, e);
                    else put(sh, sl, o, base[(size_t)j * q + r], 0.0);
                }
            }
        }
}

// Builds every table of the handle; c->{batch,k,n,bc,opts} are set by the caller.
mofem_status mofem_build(mofem_ctx* c, const mofem_profile* g1, const mofem_profile* g2,
                         const double* gamma, cudaStream_t st) {
    const int n = c->n, B = c->batch;
    HostTables H;
    MOFEM_TRY(build_host_tables(B, c->k, n, c->bc, c->opts, g1, g2, gamma, H));
    c->deg = H.K;
    c->K = H.K;
    c->P = H.P;
    c->nq = H.nq;
    c->off = H.off;
    c->q = H.q;
    c->NT = H.NT;
    const int q = c->q, off = c->off;
    c->ld = ((q + 63) / 64) * 64;
    const int ld = c->ld;
    std::vector<double>& Sh = H.S;
    std::vector<double>& Th = H.T;
    std::vector<double>& Srh = H.Srh;
    std::vector<double>& Trh = H.Trh;
    std::vector<Band>& E1s = H.E1s;
    std::vector<Band>& E2s = H.E2s;
    Band& Mt = H.Mt;
    Band& Kt = H.Kt;

    // --- double-float copies of the plain tables (residual updates, before the row-sum form)
    {
        auto split = [&](const std::vector<double>& h, float** d) -> mofem_status {
            std::vector<float> two(2 * h.size());
            for (size_t i = 0; i < h.size(); ++i) {
                const float hi = (float)h[i];
                two[i] = hi;
                two[h.size() + i] = (float)(h[i] - (double)hi);
            }
            MOFEM_TRY(dev_alloc(d, two.size()));
            MOFEM_CUDA_TRY(cudaMemcpy(*d, two.data(), two.size() * sizeof(float), cudaMemcpyHostToDevice));
            return MOFEM_OK;
        };
        MOFEM_TRY(split(Sh, &c->Sdf));   // [hi | lo] planes of [batch][NT][P][q]
        MOFEM_TRY(split(Th, &c->Tdf));   // [hi | lo] planes of [NT][P][q]
        MOFEM_TRY(split(Srh, &c->Srdf)); // [hi | lo] planes of [batch][P][q] (right-hand side)
        MOFEM_TRY(split(Trh, &c->Trdf)); // [hi | lo] planes of [P][q]
    }
    // --- double-float difference-form tables (residual of a step from zero) -------------
    {
        std::vector<float> Sd, Td;
        build_dd_tables(Sh, Th, B, c->NT, c->P, c->K, q, Sd, Td);
        MOFEM_TRY(dev_alloc(&c->Sdd, Sd.size()));
        MOFEM_CUDA_TRY(cudaMemcpy(c->Sdd, Sd.data(), Sd.size() * sizeof(float), cudaMemcpyHostToDevice));
        MOFEM_TRY(dev_alloc(&c->Tdd, Td.size()));
        MOFEM_CUDA_TRY(cudaMemcpy(c->Tdd, Td.data(), Td.size() * sizeof(float), cudaMemcpyHostToDevice));
    }

    // --- upload tables (difference form: row sum in the diagonal slot) -------------
    auto rowsum_one = [&](double* base) {
        for (int r = 0; r < q; ++r) {
            double sum = 0.0;
            for (int j = 0; j < c->P; ++j) sum += base[(size_t)j * q + r];
            base[(size_t)c->K * q + r] = sum;
        }
    };
    // T tables: every t-pass runs in difference form.  S tables: only the terms
    // whose s-factor is stiffness- or convection-like (the apply kernel's mask:
    // terms 0,3,4 of the five-term operator, 0,4,5,6,7 of the eight-term one).
    const unsigned smask = c->NT == 5 ? 0x19u : 0xF1u;
    for (int i = 0; i < B; ++i)
        for (int t = 0; t < c->NT; ++t)
            if ((smask >> t) & 1u) rowsum_one(Sh.data() + ((size_t)i * c->NT + t) * c->P * q);
    for (int t = 0; t < c->NT; ++t) rowsum_one(Th.data() + (size_t)t * c->P * q);
    rowsum_one(Trh.data());
    for (int r = 0; r < n; ++r) {   // untrimmed t-mass: row sum in the diagonal slot as well
        double sum = 0.0;
        for (int j = 0; j < c->P; ++j) sum += H.Tmf[(size_t)j * n + r];
        H.Tmf[(size_t)c->K * n + r] = sum;
    }
    std::vector<float> tmp;
    auto up64 = [&](double** d, const std::vector<double>& h) -> mofem_status {
        MOFEM_TRY(dev_alloc(d, h.size()));
        MOFEM_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
        return MOFEM_OK;
    };
    auto up32 = [&](float** d, const std::vector<double>& h) -> mofem_status {
        tmp.assign(h.begin(), h.end());
        MOFEM_TRY(dev_alloc(d, h.size()));
        MOFEM_CUDA_TRY(cudaMemcpy(*d, tmp.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
        return MOFEM_OK;
    };
    MOFEM_TRY(up64(&c->S64, Sh));
    MOFEM_TRY(up32(&c->S32, Sh));
    MOFEM_TRY(up64(&c->T64, Th));
    MOFEM_TRY(up32(&c->T32, Th));
    MOFEM_TRY(up64(&c->Sr64, Srh));
    MOFEM_TRY(up64(&c->Smf64, H.Smf));
    MOFEM_TRY(up64(&c->Tmf64, H.Tmf));
    {   // FP32 coefficient rows of the packed apply: [batch][q][W]
        const int ntp = c->NT * c->P, K = c->K, P = c->P;
        const int W = apply_s_row_floats(c->K, c->NT);
        c->s_row = W;
        std::vector<float> s2((size_t)B * q * W, 0.f);
        if (!apply_push_layout()) {   // S rows: coefficient e = t*P + j of row r at e
            for (int i = 0; i < B; ++i)
                for (int e = 0; e < ntp; ++e)
                    for (int r = 0; r < q; ++r) s2[((size_t)i * q + r) * W + e] = (float)Sh[((size_t)i * ntp + e) * q + r];
        } else {
            // push form, row g = input row g.  Difference term t: slot p < 2K is the
            // coefficient of delta[g-1] = W[g] - W[g-1] in output row j = g - K + p,
            // a_j(d) = sum_{m > d} S[j][j+m] (d >= 0) or -sum_{m <= d} S[j][j+m] (d < 0) with
            // d = K - 1 - p; slot 2K the row sum of row g.  Plain term: slot p is S[j][g].
            // Sums in FP64, one rounding.
            for (int i = 0; i < B; ++i)
                for (int t = 0; t < c->NT; ++t) {
                    const double* St = Sh.data() + ((size_t)i * c->NT + t) * P * q;   // [slot][row]
                    auto s = [&](int j, int m) -> double {   // entry (j, j + m) of the banded matrix
                        if (j < 0 || j >= q || j + m < 0 || j + m >= q) return 0.0;
                        return St[(size_t)(m + K) * q + j];
                    };
                    const bool diff = (smask >> t) & 1u;
                    for (int g = 0; g < q; ++g) {
                        float* row = s2.data() + ((size_t)i * q + g) * W + t * P;
                        if (diff) {
                            for (int p = 0; p < 2 * K; ++p) {
                                const int j = g - K + p, dd = K - 1 - p;
                                double a = 0.0;
                                if (j >= 0 && j < q) {
                                    if (dd >= 0)
                                        for (int m = dd + 1; m <= K; ++m) a += s(j, m);
                                    else
                                        for (int m = -K; m <= dd; ++m) a -= s(j, m);
                                }
                                row[p] = (float)a;
                            }
                            row[2 * K] = (float)St[(size_t)K * q + g];
                        } else {
                            for (int p = 0; p <= 2 * K; ++p) {
                                const int j = g - K + p;
                                row[p] = (float)s(j, g - j);
                            }
                        }
                    }
                }
        }
        MOFEM_TRY(dev_alloc(&c->Srow32, s2.size()));
        MOFEM_CUDA_TRY(cudaMemcpy(c->Srow32, s2.data(), s2.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    MOFEM_TRY(up64(&c->Tr64, Trh));

    // --- generalized eigendecompositions (FP64, cuSOLVER sygvd) -----------------
    cusolverDnHandle_t sol = nullptr;
    if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS) {
        mofem_set_last_error("cusolverDnCreate failed", __FILE__, __LINE__);
        return MOFEM_ERR_CUDA;
    }
    cusolverDnSetStream(sol, st);
    mofem_status result = MOFEM_OK;
    double *dA = nullptr, *dB = nullptr, *dW = nullptr, *work = nullptr;
    int* dinfo = nullptr;
    std::vector<double> hA, hB;
    int lwork = 0;
    do {
        if ((result = dev_alloc(&dA, (size_t)q * q)) != MOFEM_OK) break;
        if ((result = dev_alloc(&dB, (size_t)q * q)) != MOFEM_OK) break;
        if ((result = dev_alloc(&dW, (size_t)q)) != MOFEM_OK) break;
        if ((result = dev_alloc(&dinfo, 1)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->Q1_64, (size_t)B * q * ld)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->Q2_64, (size_t)q * ld)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->lam64, (size_t)B * ld)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->mu64, (size_t)ld)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->lam32, (size_t)B * ld)) != MOFEM_OK) break;
        if ((result = dev_alloc(&c->mu32, (size_t)ld)) != MOFEM_OK) break;
        if (cudaMemsetAsync(c->Q1_64, 0, sizeof(double) * (size_t)B * q * ld, st) != cudaSuccess ||
            cudaMemsetAsync(c->Q2_64, 0, sizeof(double) * (size_t)q * ld, st) != cudaSuccess) {
            result = MOFEM_ERR_CUDA;
            break;
        }
        if (cusolverDnDsygvd_bufferSize(sol, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                        CUBLAS_FILL_MODE_LOWER, q, dA, q, dB, q, dW, &lwork) !=
            CUSOLVER_STATUS_SUCCESS) {
            result = MOFEM_ERR_EIG;
            break;
        }
        if ((result = dev_alloc(&work, (size_t)lwork)) != MOFEM_OK) break;

        // one pencil: A x = lambda B x; dA <- eigenvectors (column-major), dW <- eigenvalues
        auto solve_pencil = [&](const Band& Am, const Band& Bm, double* Qout, double* lamout) -> mofem_status {
            dense_trimmed(Am, q, off, hA);
            dense_trimmed(Bm, q, off, hB);
            MOFEM_CUDA_TRY(cudaMemcpyAsync(dA, hA.data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, st));
            MOFEM_CUDA_TRY(cudaMemcpyAsync(dB, hB.data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, st));
            if (cusolverDnDsygvd(sol, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, q,
                                 dA, q, dB, q, dW, work, lwork, dinfo) != CUSOLVER_STATUS_SUCCESS)
                return MOFEM_ERR_EIG;
            int hinfo = 0;
            MOFEM_CUDA_TRY(cudaMemcpyAsync(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
            MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
            if (hinfo != 0) {
                mofem_set_last_error("sygvd info != 0", __FILE__, __LINE__);
                return MOFEM_ERR_EIG;
            }
            // column-major eigenvectors = row-major Q^T (row i = eigenvector i);
            // transpose into row-major Q[a][i] with leading dimension ld.
            MOFEM_TRY(launch_transpose64(dA, 0, Qout, 0, q, ld, 1, st));
            MOFEM_CUDA_TRY(cudaMemcpyAsync(lamout, dW, sizeof(double) * q, cudaMemcpyDeviceToDevice, st));
            return MOFEM_OK;
        };
        // t-pencil (shared): K_t x = mu M_t x (product form: (K_t + K_t[t^2]) x = mu x)
        if ((result = solve_pencil(H.F2, H.F1, c->Q2_64, c->mu64)) != MOFEM_OK) break;
        c->div_product = (c->opts.pencil == MOFEM_PENCIL_PRODUCT || c->opts.pencil == MOFEM_PENCIL_PARABOLIC ||
                          c->opts.pencil == MOFEM_PENCIL_AUA)
                             ? 1
                             : 0;
        for (int i = 0; i < B && result == MOFEM_OK; ++i)
            result = solve_pencil(E1s[i], E2s[i], c->Q1_64 + (size_t)i * q * ld, c->lam64 + (size_t)i * ld);
        if (result != MOFEM_OK) break;
        // pad eigenvalue tails with 1 (padded rows/columns of Q are zero)
        std::vector<double> pad1(ld - q, 1.0);
        if (ld > q) {
            for (int i = 0; i < B; ++i)
                if (cudaMemcpyAsync(c->lam64 + (size_t)i * ld + q, pad1.data(), sizeof(double) * (ld - q),
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)
                    result = MOFEM_ERR_CUDA;
            if (cudaMemcpyAsync(c->mu64 + q, pad1.data(), sizeof(double) * (ld - q), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
                result = MOFEM_ERR_CUDA;
        }
        if (result != MOFEM_OK) break;
        result = launch_convert(c->lam64, 1, ld, ld, c->lam32, 0, ld, ld, 1, ld, B, st);
        if (result != MOFEM_OK) break;
        result = launch_convert(c->mu64, 1, ld, ld, c->mu32, 0, ld, ld, 1, ld, 1, st);
        if (result != MOFEM_OK) break;
        if (cudaStreamSynchronize(st) != cudaSuccess) result = MOFEM_ERR_CUDA;
    } while (0);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dW);
    cudaFree(work);
    cudaFree(dinfo);
    cusolverDnDestroy(sol);
    return result;
}

void mofem_free(mofem_ctx* c) {
    void* ptrs[] = {c->Smf64, c->Tmf64, c->U64m, c->S64, c->S32, c->Srow32, c->Sdf, c->Tdf, c->Sdd, c->Tdd, c->Srdf, c->Trdf, c->T64, c->T32, c->Sr64, c->Tr64, c->Q1_64, c->Q2_64, c->lam64, c->mu64,
                    c->lam32, c->mu32, c->w64, c->w32, c->Bm64, c->R64, c->d_part, c->d_sc, c->d_status,
                    c->d_red};
    for (void* p : ptrs) cudaFree(p);
    for (auto& t : c->tc) {
        void* tp[] = {t.Q1, t.Q1T, t.Q2, t.Q2T, t.Rop, t.X1T, t.WT, t.Y, t.panel_cnt};
        for (void* p : tp) cudaFree(p);
    }
    for (int i = 0; i < 3; ++i) {
        if (c->it_graph[i]) cudaGraphExecDestroy(c->it_graph[i]);
        if (c->loop_graph[i]) cudaGraphExecDestroy(c->loop_graph[i]);
    }
    if (c->cublas) cublasDestroy(c->cublas);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
}

// Host-only view of the setup tables (no device work): used to check the
// assembly on machines without a GPU.  Arrays may be NULL; sizes:
// S [NT][P][q], T [NT][P][q], Srh [P][q], Trh [P][q] with NT <= 8, P = 2*max(k,1)+1.
extern "C" mofem_status mofem_host_tables(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                                          double gamma, mofem_bc bc, const mofem_opts* opts, int* n_terms, int* q_out,
                                          double* S, double* T, double* Srh, double* Trh) {
    if (!g1 || !g2 || k < 0 || k > 4 || n_nodes < 3) return MOFEM_ERR_INVALID_ARG;
    const int d = k == 0 ? 1 : k;
    if ((n_nodes - 1) % d != 0) return MOFEM_ERR_INVALID_ARG;
    mofem_opts o{};
    if (opts) o = *opts;
    HostTables H;
    MOFEM_TRY(build_host_tables(1, k, n_nodes, bc, o, g1, g2, &gamma, H));
    if (n_terms) *n_terms = H.NT;
    if (q_out) *q_out = H.q;
    if (S) std::memcpy(S, H.S.data(), H.S.size() * sizeof(double));
    if (T) std::memcpy(T, H.T.data(), H.T.size() * sizeof(double));
    if (Srh) std::memcpy(Srh, H.Srh.data(), H.Srh.size() * sizeof(double));
    if (Trh) std::memcpy(Trh, H.Trh.data(), H.Trh.size() * sizeof(double));
    return MOFEM_OK;
}

extern "C" mofem_status mofem_host_dd_tables(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                                             double gamma, mofem_bc bc, const mofem_opts* opts, float* S, float* T) {
    if (!g1 || !g2 || k < 0 || k > 4 || n_nodes < 3) return MOFEM_ERR_INVALID_ARG;
    const int d = k == 0 ? 1 : k;
    if ((n_nodes - 1) % d != 0) return MOFEM_ERR_INVALID_ARG;
    mofem_opts o{};
    if (opts) o = *opts;
    HostTables H;
    MOFEM_TRY(build_host_tables(1, k, n_nodes, bc, o, g1, g2, &gamma, H));
    std::vector<float> Sd, Td;
    build_dd_tables(H.S, H.T, 1, H.NT, H.P, H.K, H.q, Sd, Td);
    if (S) std::memcpy(S, Sd.data(), Sd.size() * sizeof(float));
    if (T) std::memcpy(T, Td.data(), Td.size() * sizeof(float));
    return MOFEM_OK;
}
