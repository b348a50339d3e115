// Host-side initialisation of a cell (Sec. 2.5 "initialisation"): validation,
// turn node sets and face lists, radial eigenbases of the separable solvers,
// unit fields and Z_vac, the network inverse and the first-cycle state.
#include "pp_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>

namespace pp {

using cd = std::complex<double>;

// ---------------------------------------------------------------- linear algebra
// cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major);
// returns eigenvalues in w and eigenvectors as the columns of V
static void jacobi_eig(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double norm = 0;
    for (double v : A) norm += v * v;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-30 * norm) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {      // columns p, q
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {      // rows p, q
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Gauss-Jordan inverse with partial pivoting; returns false if singular
template <typename T>
static bool invert(std::vector<T>& A, int n) {
    std::vector<T> I((size_t)n * n, T(0));
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = T(1);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
        if (std::abs(A[(size_t)piv * n + c]) == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
                std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
            }
        T d = A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            A[(size_t)c * n + k] /= d;
            I[(size_t)c * n + k] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            T f = A[(size_t)r * n + c];
            if (f == T(0)) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    A = I;
    return true;
}

// generalised symmetric-definite radial problem T v = mu D v, D diagonal > 0
static void radial_basis(const std::vector<double>& T, const std::vector<double>& D, int M,
                         std::vector<double>& mu, std::vector<double>& Vout) {
    std::vector<double> S((size_t)M * M);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
            S[(size_t)i * M + j] = T[(size_t)i * M + j] / std::sqrt(D[i] * D[j]);
    std::vector<double> W;
    jacobi_eig(S, M, mu, W);
    Vout.resize((size_t)M * M);
    for (int j = 0; j < M; ++j)
        for (int m = 0; m < M; ++m) Vout[(size_t)j * M + m] = W[(size_t)j * M + m] / std::sqrt(D[j]);
}

template <typename T>
static T* upload(Cell* c, const std::vector<double>& h) {
    T* d = c->alloc<T>(h.size());
    if (!d) return nullptr;
    std::vector<T> tmp(h.begin(), h.end());
    cudaMemcpy(d, tmp.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
    return d;
}

// Thomas factors of a_i x_{i-1} + d_i x_i + c_i x_{i+1} per mode (row-major [row][mode])
static void thomas_factors(const std::vector<double>& lo, const std::vector<double>& up,
                           const std::vector<double>& diag, int rows, int M, std::vector<double>& cp,
                           std::vector<double>& invd) {
    cp.assign((size_t)rows * M, 0.0);
    invd.assign((size_t)rows * M, 0.0);
    for (int m = 0; m < M; ++m) {
        double cprev = 0;
        for (int i = 0; i < rows; ++i) {
            double den = diag[(size_t)i * M + m] - (i ? lo[i] * cprev : 0.0);
            invd[(size_t)i * M + m] = 1.0 / den;
            cprev = (i + 1 < rows) ? up[i] / den : 0.0;
            cp[(size_t)i * M + m] = cprev;
        }
    }
}

// ---------------------------------------------------------------- cross sections (FP64)
static void sigma_e64(double x, double& el, double& ex, double& iz) {
    double y = x - 0.23, y2 = y * y;
    el = (0.1 + 14.0 * y2 / (y2 + 4.0)) / (1.0 + x / 50.0);
    double ye = x - 11.55;
    ex = (x > 11.55) ? 1.2 * ye / (ye * ye / 30.0 + ye + 8.0) : 0.0;
    double yi = x - 15.76;
    iz = (x > 15.76) ? 3.0 * yi / (yi * yi / 60.0 + yi + 30.0) : 0.0;
}

static void species_constants(Cell* c) {
    const pp_config& f = c->cfg;
    double n_gas = f.pressure_pa / (kKb * f.t_gas);
    // nu_max: electrons max over x = 1000 k / 100000 eV (k = 0..100000) x 1.05;
    // ions at the relative speed of a 1 keV ion (sigma g increases with g) x 1.05
    double nue = 0;
    for (int k = 0; k <= 100000; ++k) {
        double x = 1000.0 * k / 100000.0;
        double se, sx, si;
        sigma_e64(x, se, sx, si);
        double g = std::sqrt(2.0 * kQe * x / kMe);
        double nu = n_gas * 1e-20 * (se + sx + si) * g;
        nue = std::max(nue, nu);
    }
    nue *= 1.05;
    double gcap = std::sqrt(2.0 * kQe * 1000.0 / kMAr);
    double sq = std::sqrt(1000.0);
    double scx = 2.0 + 3.0 / (1.0 + sq), siso = 1.0 + 2.0 / (1.0 + sq);
    double nui = n_gas * 1e-19 * (scx + siso) * gcap * 1.05;
    for (int sp = 0; sp < 2; ++sp) {
        double q = sp == 0 ? -kQe : kQe;
        double m = sp == 0 ? kMe : kMAr;
        double nu = sp == 0 ? nue : nui;
        SpecT<double>& d = c->scd[sp];
        d.qmh = q / m * f.dt / 2.0;
        d.dtr = f.dt / c->dr;
        d.dtz = f.dt / c->dz;
        d.qw = q * f.weight[sp];
        d.numax = nu;
        d.pnull = -std::expm1(-nu * f.dt);
        d.ng = n_gas * (sp == 0 ? 1e-20 : 1e-19);
        d.ce = 0.5 * m / kQe;
        d.inv_ce = kQe / (0.5 * m);
        d.loss = 2.0 * kMe / kMAr;
        d.vth_gas = std::sqrt(kKb * f.t_gas / kMAr);
        d.qmd = q / m * f.dt;
        d.kres = q / m * f.dt * f.dt / c->dr;
        d.kzes = q / m * f.dt * f.dt / c->dz;
        d.see_g = sp == 1 ? f.see_gamma : 0.0;
        d.see_vs = sp == 1 && f.see_gamma > 0.0 ? std::sqrt(kQe * f.see_t_ev / kMe) : 0.0;
        c->chi_qm[sp] = q / m;
        SpeciesConst& s = c->sc[sp];
        s.qmh = (float)d.qmh;
        s.dtr = (float)d.dtr;
        s.dtz = (float)d.dtz;
        s.qw = (float)d.qw;
        s.numax = (float)d.numax;
        s.pnull = (float)d.pnull;
        s.ng = (float)d.ng;
        s.ce = (float)d.ce;
        s.inv_ce = (float)d.inv_ce;
        s.loss = (float)d.loss;
        s.vth_gas = (float)d.vth_gas;
        s.qmd = (float)d.qmd;
        s.kres = (float)d.kres;
        s.kzes = (float)d.kzes;
        s.see_g = (float)d.see_g;
        s.see_vs = (float)d.see_vs;
    }
}

static int on_grid(double x, double h, int* k) {
    double q = x / h;
    if (std::fabs(q - std::round(q)) > 1e-9) return 0;
    *k = (int)std::lround(q);
    return 1;
}

// The FP64 separable solver of the Helmholtz operator (Eq. helmholtz_op) on
// the interior unknowns i = 1..NZ-2, j = 1..NR-2 (E_theta = 0 on the axis and
// the outer boundaries): the radial generalised eigenbasis T v = mu D v
// (D = R) and per-mode Thomas factors in z; k2base = mu0 eps0 w^2 (0: MQS)
// times the node-row average of eps_row.
static void build_helmholtz_into(Cell* c, SepSolver<double>& s, double k2base) {
    const int NR = c->NR, rows = c->NZ - 2, MH = NR - 2;
    const double dr = c->dr, dz = c->dz;
    std::vector<double> T((size_t)MH * MH, 0.0), D(MH);
    for (int jj = 0; jj < MH; ++jj) {
        int j = jj + 1;
        double R = j * dr, bj = R + dr / 2, bm = R - dr / 2;
        T[(size_t)jj * MH + jj] = -(bj + bm) / (dr * dr) - 1.0 / R;
        if (jj + 1 < MH) T[(size_t)jj * MH + jj + 1] = bj / (dr * dr);
        if (jj > 0) T[(size_t)jj * MH + jj - 1] = bm / (dr * dr);
        D[jj] = R;
    }
    std::vector<double> mu, V;
    radial_basis(T, D, MH, mu, V);
    std::vector<double> Vf((size_t)MH * MH), Vb((size_t)MH * MH);
    for (int jj = 0; jj < MH; ++jj)
        for (int m = 0; m < MH; ++m) {
            Vf[(size_t)jj * MH + m] = D[jj] * V[(size_t)jj * MH + m];
            Vb[(size_t)m * MH + jj] = V[(size_t)jj * MH + m];
        }
    std::vector<double> lo(rows), up(rows), diag((size_t)rows * MH), cp, invd;
    for (int ii = 0; ii < rows; ++ii) {
        int i = ii + 1;
        double epsn = 0.5 * (c->eps_row[i - 1] + c->eps_row[i]);
        lo[ii] = (ii > 0) ? 1.0 / (dz * dz) : 0.0;
        up[ii] = 1.0 / (dz * dz);
        for (int m = 0; m < MH; ++m) diag[(size_t)ii * MH + m] = -2.0 / (dz * dz) + mu[m] + k2base * epsn;
    }
    thomas_factors(lo, up, diag, rows, MH, cp, invd);
    s.rows = rows;
    s.M = MH;
    s.Vf = upload<double>(c, Vf);
    s.Vb = upload<double>(c, Vb);
    s.cp = upload<double>(c, cp);
    s.invd = upload<double>(c, invd);
    s.lo = upload<double>(c, lo);
    s.t0 = c->alloc<double>((size_t)rows * MH);
    s.t1 = c->alloc<double>((size_t)rows * MH);
}

static void build_helmholtz(Cell* c, double k2base) {
    build_helmholtz_into(c, c->hs, k2base);
    c->d_hstage = c->alloc<double>((size_t)2 * (c->NZ - 2) * (c->NR - 2));
}

// Network constants at angular frequency w (Eqs. skin, zsource, blockmatrix):
// R_rf per turn, Z_source, Z_turn = Z_vac + diag(R_rf), the inverse of the
// (2N+1) network matrix, and the circ vector (zs, r_rf, c_stray).  false when
// the matrix is singular.
static bool network_constants(const Cell* c, double w, const std::vector<double>& zvac, std::vector<double>& r_rf,
                              std::vector<std::complex<double>>& Ainv, std::vector<double>& ainv,
                              std::vector<double>& ztv, std::vector<double>& circ) {
    const pp_config& f = c->cfg;
    const int N = c->nturns, NX = 2 * N + 1;
    r_rf.assign(N, 0.0);
    if (f.r_rf_override >= 0) {
        for (int k = 0; k < N; ++k) r_rf[k] = f.r_rf_override;
    } else {
        double rho = f.rho20 * (1.0 + f.alpha_cu * (f.t_coil_c - 20.0));
        double delta = std::sqrt(2.0 * rho / (w * kMu0));
        double inner = std::max(f.wire_radius - delta, 0.0);
        for (int k = 0; k < N; ++k)
            r_rf[k] = rho * 2 * kPi * f.turn_r[k] / (kPi * (f.wire_radius * f.wire_radius - inner * inner));
    }
    double xs = w * f.l_m;
    if (f.c_m > 0) xs -= 1.0 / (w * f.c_m);
    cd zs(f.r_g + f.r_m, xs);
    std::vector<cd> A((size_t)NX * NX, cd(0, 0));
    std::vector<cd> zt((size_t)N * N);
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l)
            zt[(size_t)k * N + l] = cd(zvac[2 * (k * N + l)], zvac[2 * (k * N + l) + 1]) + (k == l ? r_rf[k] : 0.0);
    A[0] = zs;
    A[1 + N] = 1.0;
    for (int k = 0; k < N; ++k) {
        int r = 1 + k;
        A[(size_t)r * NX + (k == 0 ? 0 : k)] = 1.0;          // I_in,k
        A[(size_t)r * NX + 1 + k] = -1.0;
        A[(size_t)r * NX + 1 + N + k] = cd(0, -w * f.c_stray[k]);
        int r2 = 1 + N + k;
        for (int l = 0; l < N; ++l) A[(size_t)r2 * NX + 1 + l] = -zt[(size_t)k * N + l];
        A[(size_t)r2 * NX + 1 + N + k] = 1.0;
        if (k + 1 < N) A[(size_t)r2 * NX + 1 + N + k + 1] = -1.0;
    }
    Ainv = A;
    if (!invert(Ainv, NX)) return false;
    ainv.assign(2 * NX * NX, 0.0);
    ztv.assign(2 * N * N, 0.0);
    circ.assign(2 + 2 * N, 0.0);
    for (int q = 0; q < NX * NX; ++q) {
        ainv[2 * q] = Ainv[q].real();
        ainv[2 * q + 1] = Ainv[q].imag();
    }
    for (int q = 0; q < N * N; ++q) {
        ztv[2 * q] = zt[q].real();
        ztv[2 * q + 1] = zt[q].imag();
    }
    circ[0] = zs.real();
    circ[1] = zs.imag();
    for (int k = 0; k < N; ++k) {
        circ[2 + k] = r_rf[k];
        circ[2 + N + k] = f.c_stray[k];
    }
    return true;
}

static int fail(const char* msg) {
    set_error(msg);
    return PP_E_CONFIG;
}

// ---------------------------------------------------------------- setup
int setup_cell(Cell* c) {
    pp_config& f = c->cfg;
    if (f.nr < 2 || f.nz < 4 || f.r_max <= 0 || f.z_max <= 0) return fail("grid sizes must be positive");
    if (f.nr + 1 > kMaxNR) return fail("nr exceeds the supported radial node count");
    if (f.nz - 1 > (1 << kMaxPcrLevels)) return fail("nz exceeds the supported axial node count");
    if (f.n_turns < 1 || f.n_turns > PP_MAX_TURNS) return fail("n_turns out of range");
    if (f.freq <= 0 || f.dt <= 0) return fail("freq and dt must be positive");
    if (f.plain_fp64 != 0 && f.plain_fp64 != 1) return fail("plain_fp64 must be 0 or 1");
    if (f.implicit_es != 0 && f.implicit_es != 1) return fail("implicit_es must be 0 or 1");
    if (f.n_harmonics < 0 || f.n_harmonics > PP_MAX_HARM) return fail("n_harmonics must be in 1..PP_MAX_HARM");
    if (!(f.see_gamma >= 0.0 && f.see_gamma <= 1.0)) return fail("see_gamma must lie in [0, 1]");
    if (f.see_gamma > 0.0 && !(f.see_t_ev > 0.0 && std::isfinite(f.see_t_ev)))
        return fail("see_t_ev must be positive");
    if (f.see_gamma > 0.0 && f.weight[0] != f.weight[1])
        return fail("secondary emission needs equal macro weights of electrons and ions");
    if (f.particle_weights != 0 && f.particle_weights != 1) return fail("particle_weights must be 0 or 1");
    if (f.sm_every < 0) return fail("sm_every must be >= 0");
    if (f.sm_every > 0 && !(f.sm_min >= 1 && f.sm_min <= f.sm_target && f.sm_target <= f.sm_max))
        return fail("split-merge needs 1 <= sm_min <= sm_target <= sm_max");
    c->implicit = f.implicit_es == 1;
    c->see = f.see_gamma > 0.0;
    c->sm_every = f.sm_every;
    c->sm_target = f.sm_target;
    c->sm_min = f.sm_min;
    c->sm_max = f.sm_max;
    c->weighted = f.particle_weights == 1 || f.sm_every > 0;
    c->nr = f.nr;
    c->nz = f.nz;
    c->NR = f.nr + 1;
    c->NZ = f.nz + 1;
    c->nnodes = c->NR * c->NZ;
    c->dr = f.r_max / f.nr;
    c->dz = f.z_max / f.nz;
    c->omega = 2.0 * kPi * f.freq;
    c->nturns = f.n_turns;
    // Eq. nrf and Eq. phaseclosure
    c->n_rf = (int)std::lround(1.0 / (f.freq * f.dt));
    if (!(std::fabs(f.freq * f.dt * c->n_rf - 1.0) < 1e-10)) return fail("phase closure violated: |f dt N_RF - 1| >= 1e-10");
    if (!on_grid(f.z_win_lo, c->dz, &c->i_win) || !on_grid(f.z_win_hi, c->dz, &c->i_win_hi))
        return fail("window planes must lie on grid lines");
    if (c->i_win < 2 || c->i_win_hi <= c->i_win || c->i_win_hi >= f.nz) return fail("window slab out of range");
    if (f.weight[0] <= 0 || f.weight[1] <= 0) return fail("macroparticle weights must be positive");
    if (f.capacity[0] < 1 || f.capacity[1] < 1) return fail("capacities must be positive");
    if (f.capacity[0] > 0x7fffffff - kChunk || f.capacity[1] > 0x7fffffff - kChunk) return fail("capacity too large");
    if (f.sort_every[0] < 1 || f.sort_every[1] < 1) return fail("sort_every must be >= 1");
    if (f.alpha <= 0 || f.alpha > 1) return fail("relaxation factor must be in (0, 1]");
    if (f.poisson_tol <= 0) f.poisson_tol = 1e-10;
    if (f.poisson_max_iter < 1) f.poisson_max_iter = 4;
    const int NR = c->NR, NZ = c->NZ, N = c->nturns;
    const double dr = c->dr, dz = c->dz;

    // ---- permittivity per cell row (the slab spans the full radius)
    c->eps_row.assign(f.nz, 1.0);
    for (int i = c->i_win; i < c->i_win_hi; ++i) c->eps_row[i] = f.eps_win;

    // ---- turn node sets (Eq. shape): nodes within the wire disc, else nearest
    std::vector<int> owner(c->nnodes, -1);
    c->turn_nodes.assign(N, {});
    for (int k = 0; k < N; ++k) {
        std::vector<int>& nodes = c->turn_nodes[k];
        double rk = f.turn_r[k];
        for (int i = 1; i <= NZ - 2; ++i)
            for (int j = 0; j <= NR - 2; ++j) {
                double d2 = (j * dr - rk) * (j * dr - rk) + (i * dz - f.z_coil) * (i * dz - f.z_coil);
                if (d2 <= f.wire_radius * f.wire_radius) nodes.push_back(i * NR + j);
            }
        if (nodes.empty()) {
            double best = 1e300;
            int bn = -1;
            for (int i = 1; i <= NZ - 2; ++i)
                for (int j = 0; j <= NR - 2; ++j) {
                    double d2 = (j * dr - rk) * (j * dr - rk) + (i * dz - f.z_coil) * (i * dz - f.z_coil);
                    if (d2 < best) {
                        best = d2;
                        bn = i * NR + j;
                    }
                }
            nodes.push_back(bn);
        }
        for (int n : nodes) {
            if (owner[n] >= 0) return fail("a conductor node belongs to two turns");
            if (n / NR <= c->i_win) return fail("a turn reaches into the plasma region");
            owner[n] = k;
        }
        if (f.winding[k] != 1 && f.winding[k] != -1) return fail("winding signs must be +1 or -1");
        double sum = 0;
        for (size_t q = 0; q < nodes.size(); ++q) sum += f.winding[k] / (nodes.size() * dz * dr) * dz * dr;
        if (std::fabs(sum - f.winding[k]) > 1e-12) return fail("shape normalisation failed");
    }
    std::vector<int> tn_node, tn_int, tn_k;
    std::vector<double> gk_val;
    const int rows = NZ - 2, M = NR - 1;
    for (int k = 0; k < N; ++k)
        for (int n : c->turn_nodes[k]) {
            tn_node.push_back(n);
            tn_int.push_back((n / NR - 1) * M + (n % NR));
            tn_k.push_back(k);
            gk_val.push_back(f.winding[k] / (c->turn_nodes[k].size() * dz * dr));
        }
    c->ntn = (int)tn_node.size();
    if (c->ntn > kMaxCapNodes) return fail("too many turn nodes for the capacitance correction");
    // the step's field preparation imposes the turn potentials while it reads
    // the potential of node rows 0..i_win+1: the coil must lie above them
    for (int n : tn_node)
        if (n / NR <= c->i_win + 1) return fail("coil turn nodes must lie above the first row over the window");
    if (NR - 1 > 512) return fail("nr exceeds the radial unknowns supported by the Poisson solver");
    std::vector<signed char> mask(c->nnodes, -1);
    for (int t = 0; t < c->ntn; ++t) mask[tn_node[t]] = (signed char)tn_k[t];

    // ---- faces of Eq. facecharge with the areas of Eq. areas
    std::vector<int> ft, fnb, fk;
    std::vector<double> fc;
    auto area_z = [&](int j) { return j == 0 ? kPi * (dr / 2) * (dr / 2) : 2 * kPi * (j * dr) * dr; };
    for (int k = 0; k < N; ++k)
        for (int n : c->turn_nodes[k]) {
            int i = n / NR, j = n % NR;
            const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
            for (int q = 0; q < 4; ++q) {
                if (j == 0 && dj[q] == -1) continue;
                int ii = i + di[q], jj = j + dj[q];
                if (ii < 0 || ii >= NZ || jj < 0 || jj >= NR) continue;
                int nb = ii * NR + jj;
                if (owner[nb] == k) continue;
                double A, d, eps;
                if (di[q] != 0) {
                    A = area_z(j);
                    d = dz;
                    eps = c->eps_row[di[q] > 0 ? i : i - 1];
                } else {
                    A = 2 * kPi * (j * dr + dj[q] * dr / 2) * dz;
                    d = dr;
                    eps = 0.5 * (c->eps_row[i - 1] + c->eps_row[i]);
                }
                ft.push_back(n);
                fnb.push_back(nb);
                fk.push_back(k);
                fc.push_back(kEps0 * eps * A / d);
            }
        }
    c->nfaces = (int)ft.size();

    // ---- node weighting volumes (V = int S dV) of the plasma rows
    std::vector<double> vol(c->nnodes, 0.0);
    for (int i = 0; i <= c->i_win; ++i)
        for (int j = 0; j < NR; ++j) {
            double vr = 2 * kPi * (j * dr) * dr;
            if (j == 0) vr = kPi * dr * dr / 3.0;
            if (j == NR - 1) vr = kPi * (f.r_max * dr - dr * dr / 3.0);
            double vz = (i == 0 || i == c->i_win) ? dz / 2.0 : dz;
            vol[i * NR + j] = vz * vr;
        }

    // ---- per-column FV factors of the Poisson operator divided by 2 pi
    std::vector<double> az(NR), arp(NR), arm(NR), Rn(NR);
    for (int j = 0; j < NR; ++j) {
        Rn[j] = j * dr;
        az[j] = (j == 0 ? dr * dr / 8.0 : j * dr * dr) / dz;
        arp[j] = (j * dr + dr / 2) * dz / dr;
        arm[j] = (j == 0) ? 0.0 : (j * dr - dr / 2) * dz / dr;
    }

    // ---- cell / nr by multiply-high and shift, verified for every plasma cell
    {
        uint32_t d = (uint32_t)f.nr, s = 0;
        while ((2u << s) <= d) ++s;                       // s = floor(log2 d)
        if ((d & (d - 1)) == 0) --s;                      // powers of two: m = 2^31
        uint64_t m = (((uint64_t)1 << (32 + s)) + d - 1) / d;
        if (m >> 32) return fail("no 32-bit division multiplier for nr");
        uint32_t ncell = (uint32_t)(c->i_win * f.nr);
        for (uint32_t q = 0; q < ncell; ++q)
            if ((uint32_t)(((uint64_t)q * m) >> 32 >> s) != q / d) return fail("division multiplier check failed");
        c->div_magic = (uint32_t)m;
        c->div_shift = s;
    }

    // ---- allocations (particle storage padded to whole staging chunks)
    c->fp64 = f.plain_fp64 != 0;
    for (int sp = 0; sp < 2; ++sp) {
        c->cap[sp] = f.capacity[sp];
        for (int b = 0; b < 2; ++b) {
            size_t n = (size_t)((c->cap[sp] + kChunk - 1) / kChunk) * kChunk;
            bool ok;
            if (c->fp64) {
                PBuf<double>& p = c->pd[sp][b];
                p.cell = c->alloc<uint32_t>(n);
                p.dr = c->alloc<double>(n);
                p.dz = c->alloc<double>(n);
                p.vr = c->alloc<double>(n);
                p.vt = c->alloc<double>(n);
                p.vz = c->alloc<double>(n);
                p.uid = c->alloc<uint32_t>(n);
                p.w = c->weighted ? c->alloc<double>(n) : nullptr;
                ok = p.cell && p.dr && p.dz && p.vr && p.vt && p.vz && p.uid && (p.w || !c->weighted);
                c->pb[sp][b] = ParticleBuf{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            } else {
                ParticleBuf& p = c->pb[sp][b];
                p.cell = c->alloc<uint32_t>(n);
                p.dr = c->alloc<float>(n);
                p.dz = c->alloc<float>(n);
                p.vr = c->alloc<float>(n);
                p.vt = c->alloc<float>(n);
                p.vz = c->alloc<float>(n);
                p.uid = c->alloc<uint32_t>(n);
                p.w = c->weighted ? c->alloc<float>(n) : nullptr;
                ok = p.cell && p.dr && p.dz && p.vr && p.vt && p.vz && p.uid && (p.w || !c->weighted);
                c->pd[sp][b] = PBuf<double>{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            }
            if (!ok) {
                set_error("cudaMalloc failed for the particle store");
                return PP_E_CUDA;
            }
        }
    }
    // ionisation events of one step: at least kEventMin, else 1/64 of the
    // electron capacity (a step that creates more than 1.5 % of the
    // population in pairs is far outside any regime the method resolves)
    {
        int64_t ec = (c->cap[0] + 63) / 64;
        ec = ec < kEventMin ? kEventMin : ec;
        ec = ec > (int64_t)1 << 22 ? (int64_t)1 << 22 : ec;
        c->event_cap = (int)((ec + kAppendThreads - 1) / kAppendThreads * kAppendThreads);
    }
    c->d_ev_perm = c->alloc<uint32_t>(c->event_cap);
    if (c->fp64) {
        c->d_events64 = c->alloc<EventT<double>>(c->event_cap);
        c->d_F64 = c->alloc<double>((size_t)c->i_win * f.nr * 20);
        c->d_rho64 = c->alloc<double>((size_t)2 * c->nnodes);
        c->d_jm64 = c->alloc<double>(c->nnodes);
    }
    c->d_nslot = c->alloc<int>(2);
    c->d_next_uid = c->alloc<uint32_t>(2);
    c->d_hist = c->alloc<uint32_t>((size_t)c->i_win * c->nr + 2);
    c->d_events = c->alloc<Event>(c->event_cap);
    if (c->sm_every > 0) {
        const size_t ncell = (size_t)c->i_win * c->nr;
        const int64_t capmax = c->cap[0] > c->cap[1] ? c->cap[0] : c->cap[1];
        c->d_sm_cnt = c->alloc<uint32_t>(ncell + 2);
        c->d_sm_start = c->alloc<uint32_t>(ncell + 1);
        c->d_sm_cursor = c->alloc<uint32_t>(ncell + 1);
        c->d_sm_soff = c->alloc<uint32_t>(ncell + 1);
        c->d_sm_list = c->alloc<int>(ncell + 1);
        c->d_sm_perm = c->alloc<uint32_t>((size_t)capmax);
        if (!c->d_sm_cnt || !c->d_sm_start || !c->d_sm_cursor || !c->d_sm_soff || !c->d_sm_list || !c->d_sm_perm) {
            set_error("cudaMalloc failed for the split-merge buffers");
            return PP_E_CUDA;
        }
    }
    c->d_phi = c->alloc<double>(c->nnodes);
    c->d_F = c->alloc<float>((size_t)c->i_win * c->nr * 20);
    c->d_rho = c->alloc<float>((size_t)2 * c->nnodes);
    c->d_jm = c->alloc<float>(c->nnodes);
    c->d_win = c->alloc<double>(c->nnodes);
    c->d_vol = upload<double>(c, vol);
    {
        // susceptibility weight per node: chi = (q_e/m_e rho_e + q_i/m_i rho_i) * chiw with
        // chiw = dt^2 / (eps0 V eps_r), eps_r the mean of the node's adjacent cells (Sec. 2.3)
        std::vector<double> chiw(c->nnodes, 0.0);
        for (int i = 0; i <= c->i_win; ++i) {
            const double eps_n = i == 0 ? c->eps_row[0] : 0.5 * (c->eps_row[i - 1] + c->eps_row[i]);
            for (int j = 0; j < NR; ++j) {
                const double v = vol[i * NR + j];
                chiw[i * NR + j] = v > 0 ? f.dt * f.dt / (kEps0 * v * eps_n) : 0.0;
            }
        }
        c->d_chiw = upload<double>(c, chiw);
    }
    c->d_Ec = c->alloc<double>(c->nnodes);
    c->d_Ess = c->alloc<double>(c->nnodes);
    c->d_Ecp = c->alloc<double>(c->nnodes);
    c->d_Essp = c->alloc<double>(c->nnodes);
    c->d_Ecp_new = c->alloc<double>(c->nnodes);
    c->d_Essp_new = c->alloc<double>(c->nnodes);
    c->d_Br = c->alloc<double>((size_t)4 * c->nnodes);
    c->d_U = c->alloc<double>((size_t)N * c->nnodes);
    c->d_Jc = c->alloc<double>(c->nnodes);
    c->d_Js = c->alloc<double>(c->nnodes);
    c->d_Jc_c = c->alloc<double>(c->nnodes);
    c->d_Js_c = c->alloc<double>(c->nnodes);
    c->d_eps_row = upload<double>(c, c->eps_row);
    c->d_az = upload<double>(c, az);
    c->d_arp = upload<double>(c, arp);
    c->d_arm = upload<double>(c, arm);
    c->d_R = upload<double>(c, Rn);
    {
        std::vector<double> tmp;
        c->d_face_c = upload<double>(c, fc);
        c->d_face_t = c->alloc<int>(ft.size());
        c->d_face_nb = c->alloc<int>(fnb.size());
        c->d_face_k = c->alloc<int>(fk.size());
        cudaMemcpy(c->d_face_t, ft.data(), sizeof(int) * ft.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_face_nb, fnb.data(), sizeof(int) * fnb.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_face_k, fk.data(), sizeof(int) * fk.size(), cudaMemcpyHostToDevice);
        c->d_tn_node = c->alloc<int>(c->ntn);
        c->d_tn_int = c->alloc<int>(c->ntn);
        c->d_tn_k = c->alloc<int>(c->ntn);
        cudaMemcpy(c->d_tn_node, tn_node.data(), sizeof(int) * c->ntn, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_tn_int, tn_int.data(), sizeof(int) * c->ntn, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_tn_k, tn_k.data(), sizeof(int) * c->ntn, cudaMemcpyHostToDevice);
        c->d_gk_val = upload<double>(c, gk_val);
        c->d_turn_mask = c->alloc<signed char>(c->nnodes);
        cudaMemcpy(c->d_turn_mask, mask.data(), c->nnodes, cudaMemcpyHostToDevice);
    }
    c->d_st = c->alloc<DevState>(1);
    if (cudaMallocHost(&c->h_st, sizeof(DevState)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return PP_E_CUDA;
    }
    memset(c->h_st, 0, sizeof(DevState));
    c->d_ext_targets = c->alloc<double>(PP_MAX_TURNS);
    if (!c->d_st || !c->d_Js_c) {
        set_error("cudaMalloc failed for the field grids");
        return PP_E_CUDA;
    }

    // ---- Poisson FP32 separable solver (radial unknowns j = 0..NR-2)
    {
        std::vector<double> T((size_t)M * M, 0.0), D(M);
        for (int j = 0; j < M; ++j) {
            double bj = (j + 0.5) * dr, bm = (j > 0) ? (j - 0.5) * dr : 0.0;
            T[(size_t)j * M + j] = -(bj + bm);
            if (j + 1 < M) T[(size_t)j * M + j + 1] = bj;
            if (j > 0) T[(size_t)j * M + j - 1] = bm;
            D[j] = (j == 0) ? dr * dr / 8.0 : j * dr * dr;
        }
        std::vector<double> mu, V;
        radial_basis(T, D, M, mu, V);
        c->ps_mu = mu;
        std::vector<double> Vt((size_t)M * M);
        for (int j = 0; j < M; ++j)
            for (int m = 0; m < M; ++m) Vt[(size_t)m * M + j] = V[(size_t)j * M + m];
        std::vector<double> lo(rows), up(rows), diag((size_t)rows * M), cp, invd;
        for (int ii = 0; ii < rows; ++ii) {
            int i = ii + 1;
            double ep = c->eps_row[i], em = c->eps_row[i - 1], eb = 0.5 * (ep + em);
            lo[ii] = (ii > 0) ? em / dz : 0.0;
            up[ii] = ep / dz;
            for (int m = 0; m < M; ++m) diag[(size_t)ii * M + m] = -(ep + em) / dz + (dz / dr) * eb * mu[m];
        }
        thomas_factors(lo, up, diag, rows, M, cp, invd);
        // parallel cyclic reduction of the same per-mode systems: level l
        // (stride 2^l) maps d_i -> d_i + alpha_i d_{i-s} + gamma_i d_{i+s};
        // after the last level x_i = d_i / b_i.  The coefficients depend only
        // on the operator, so they are reduced here in FP64 once.
        {
            int L = 0;
            while ((1 << L) < rows) ++L;
            std::vector<double> al((size_t)L * rows * M), ga((size_t)L * rows * M), ib((size_t)rows * M);
            std::vector<double> a(rows), b(rows), cc(rows), a2(rows), b2(rows), c2(rows);
            for (int m = 0; m < M; ++m) {
                for (int i = 0; i < rows; ++i) {
                    a[i] = lo[i];
                    b[i] = diag[(size_t)i * M + m];
                    cc[i] = (i + 1 < rows) ? up[i] : 0.0;
                }
                for (int l = 0; l < L; ++l) {
                    int st = 1 << l;
                    for (int i = 0; i < rows; ++i) {
                        int im = i - st, ip = i + st;
                        double alpha = (im >= 0) ? -a[i] / b[im] : 0.0;
                        double gamma = (ip < rows) ? -cc[i] / b[ip] : 0.0;
                        al[((size_t)m * L + l) * rows + i] = alpha;
                        ga[((size_t)m * L + l) * rows + i] = gamma;
                        a2[i] = (im >= 0) ? alpha * a[im] : 0.0;
                        c2[i] = (ip < rows) ? gamma * cc[ip] : 0.0;
                        b2[i] = b[i] + ((im >= 0) ? alpha * cc[im] : 0.0) + ((ip < rows) ? gamma * a[ip] : 0.0);
                    }
                    a.swap(a2);
                    b.swap(b2);
                    cc.swap(c2);
                }
                for (int i = 0; i < rows; ++i) ib[(size_t)m * rows + i] = 1.0 / b[i];
            }
            c->pcr_levels = L;
            c->d_pcr_a = upload<float>(c, al);
            c->d_pcr_g = upload<float>(c, ga);
            c->d_pcr_ib = upload<float>(c, ib);
        }
        SepSolver<float>& s = c->ps;
        s.rows = rows;
        s.M = M;
        s.Vf = upload<float>(c, V);
        s.Vb = upload<float>(c, Vt);
        s.cp = upload<float>(c, cp);
        s.invd = upload<float>(c, invd);
        s.lo = upload<float>(c, lo);
        s.t0 = c->alloc<float>((size_t)rows * M);
        s.t1 = c->alloc<float>((size_t)rows * M);
        c->d_r32 = c->alloc<float>((size_t)rows * M);
        c->d_sigma = c->alloc<double>(kMaxCapNodes);
        c->d_rT = c->alloc<double>(kMaxCapNodes);
    }
    // ---- Helmholtz FP64 separable solver (radial unknowns j = 1..NR-2)
    build_helmholtz(c, f.full_helmholtz ? kMu0 * kEps0 * c->omega * c->omega : 0.0);
    if (!c->d_hstage) {
        set_error("cudaMalloc failed for the solver storage");
        return PP_E_CUDA;
    }

    species_constants(c);

    // ---- unit fields K U_k = g_k (Eq. unitfield) and Z_vac (Eq. zvac)
    std::vector<double> gk((size_t)c->nnodes, 0.0);
    std::vector<double> Uh((size_t)N * c->nnodes);
    double* d_g = c->alloc<double>(c->nnodes);
    for (int k = 0; k < N; ++k) {
        std::fill(gk.begin(), gk.end(), 0.0);
        double g = f.winding[k] / (c->turn_nodes[k].size() * dz * dr);
        for (int n : c->turn_nodes[k]) gk[n] = g;
        cudaMemcpy(d_g, gk.data(), sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
        helmholtz_solve_dev(c, d_g, c->d_U + (size_t)k * c->nnodes, kMu0 * c->omega, 0);
    }
    cudaMemcpy(Uh.data(), c->d_U, sizeof(double) * N * c->nnodes, cudaMemcpyDeviceToHost);
    c->zvac.assign(2 * N * N, 0.0);
    double zmax = 0, dmax = 0;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) {
            double s = 0;
            double g = f.winding[k] / (c->turn_nodes[k].size() * dz * dr);
            for (int n : c->turn_nodes[k]) s += g * Uh[(size_t)l * c->nnodes + n] * 2 * kPi * ((n % NR) * dr) * dz * dr;
            c->zvac[2 * (k * N + l)] = 0.0;
            c->zvac[2 * (k * N + l) + 1] = -s;        // -i * s
        }
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) {
            zmax = std::max(zmax, std::fabs(c->zvac[2 * (k * N + l) + 1]));
            dmax = std::max(dmax, std::fabs(c->zvac[2 * (k * N + l) + 1] - c->zvac[2 * (l * N + k) + 1]));
        }
    c->eps_rec = zmax > 0 ? dmax / zmax : 0.0;

    // ---- R_rf (Eq. skin), Z_source (Eq. zsource), network (Eq. blockmatrix)
    const int NX = 2 * N + 1;
    std::vector<cd> Ainv;
    std::vector<double> ainv, ztv, circ;
    if (!network_constants(c, c->omega, c->zvac, c->r_rf, Ainv, ainv, ztv, circ))
        return fail("network matrix is singular");
    c->d_Ainv = upload<double>(c, ainv);
    c->d_zturn = upload<double>(c, ztv);
    c->d_circ = upload<double>(c, circ);

    // ---- retained harmonics m = 2..M (the multiharmonic extension of
    // Sec. 4): Helmholtz operator (k^2 m^2), unit fields, Z_vac and network at
    // m w, field and accumulator storage; the harmonic states start at zero
    // (no source at m w)
    c->nharm = f.n_harmonics < 1 ? 1 : f.n_harmonics;
    if (c->nharm > 1) {
        const int nh = c->nharm - 1;
        const size_t nn = (size_t)c->nnodes;
        c->d_Uh = c->alloc<double>((size_t)nh * N * nn);
        c->d_Ech = c->alloc<double>((size_t)nh * 2 * nn);
        c->d_Ecph = c->alloc<double>((size_t)nh * 4 * nn);
        c->d_Bh = c->alloc<double>((size_t)nh * 4 * nn);
        c->d_Jh = c->alloc<double>((size_t)nh * 4 * nn);
        std::vector<double> ainvh, zth, circh;
        c->zvach.assign((size_t)nh * 2 * N * N, 0.0);
        std::vector<double> Uhh((size_t)N * nn);
        for (int h = 0; h < nh; ++h) {
            const int m = h + 2;
            const double wm = m * c->omega;
            build_helmholtz_into(c, c->hsh[h], f.full_helmholtz ? kMu0 * kEps0 * wm * wm : 0.0);
            double* Uh = c->d_Uh + (size_t)h * N * nn;
            for (int k = 0; k < N; ++k) {
                std::fill(gk.begin(), gk.end(), 0.0);
                double gv = f.winding[k] / (c->turn_nodes[k].size() * dz * dr);
                for (int n : c->turn_nodes[k]) gk[n] = gv;
                cudaMemcpy(d_g, gk.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
                helmholtz_solve_sep(c, c->hsh[h], d_g, Uh + (size_t)k * nn, kMu0 * wm, 0);
            }
            cudaMemcpy(Uhh.data(), Uh, sizeof(double) * N * nn, cudaMemcpyDeviceToHost);
            std::vector<double> zv(2 * N * N, 0.0);
            for (int k = 0; k < N; ++k)
                for (int l = 0; l < N; ++l) {
                    double sum = 0;
                    double gv = f.winding[k] / (c->turn_nodes[k].size() * dz * dr);
                    for (int n : c->turn_nodes[k]) sum += gv * Uhh[(size_t)l * nn + n] * 2 * kPi * ((n % NR) * dr) * dz * dr;
                    zv[2 * (k * N + l) + 1] = -sum;
                }
            std::copy(zv.begin(), zv.end(), c->zvach.begin() + (size_t)h * 2 * N * N);
            std::vector<cd> Ah;
            std::vector<double> rr, ai, zt, ci;
            if (!network_constants(c, wm, zv, rr, Ah, ai, zt, ci)) return fail("harmonic network matrix is singular");
            ainvh.insert(ainvh.end(), ai.begin(), ai.end());
            zth.insert(zth.end(), zt.begin(), zt.end());
            circh.insert(circh.end(), ci.begin(), ci.end());
        }
        c->d_Ainvh = upload<double>(c, ainvh);
        c->d_zturnh = upload<double>(c, zth);
        c->d_circh = upload<double>(c, circh);
    }

    // ---- x^1: zero-load network solution
    cd vg(f.v_g * std::cos(f.phase_g), f.v_g * std::sin(f.phase_g));
    DevState* h = c->h_st;
    for (int q = 0; q < NX; ++q) {
        cd x = Ainv[(size_t)q * NX + 0] * vg;
        h->x[2 * q] = x.real();
        h->x[2 * q + 1] = x.imag();
    }
    h->vg_amp = f.v_g;
    h->nharm = c->nharm;
    cudaMemcpy(c->d_st, h, sizeof(DevState), cudaMemcpyHostToDevice);
    launch_compose(c, false, 0);

    // ---- capacitance correction: Z_t = P(e_t), G = Z_T, G^-1
    {
        int K = c->ntn;
        size_t nint = (size_t)rows * M;
        c->d_Z = c->alloc<float>((size_t)K * nint);
        std::vector<float> e(nint, 0.0f);
        for (int t = 0; t < K; ++t) {
            std::fill(e.begin(), e.end(), 0.0f);
            e[tn_int[t]] = 1.0f;
            cudaMemcpy(c->d_r32, e.data(), sizeof(float) * nint, cudaMemcpyHostToDevice);
            poisson_fast_solve(c, c->d_r32, c->d_Z + (size_t)t * nint, 0);
        }
        std::vector<float> Zh((size_t)K * nint);
        cudaMemcpy(Zh.data(), c->d_Z, sizeof(float) * K * nint, cudaMemcpyDeviceToHost);
        std::vector<double> G((size_t)K * K);
        for (int t = 0; t < K; ++t)
            for (int u = 0; u < K; ++u) G[(size_t)t * K + u] = Zh[(size_t)u * nint + tn_int[t]];
        if (!invert(G, K)) return fail("capacitance matrix is singular");
        c->d_Ginv = upload<double>(c, G);
        // interleaved copy: the K corrections of one unknown are contiguous
        int Kp = (K + 3) / 4 * 4;
        std::vector<double> Zt(nint * (size_t)Kp, 0.0);
        for (size_t q = 0; q < nint; ++q)
            for (int t = 0; t < K; ++t) Zt[q * Kp + t] = Zh[(size_t)t * nint + q];
        c->ntn_pad = Kp;
        c->d_Zt = upload<float>(c, Zt);
    }
    // ---- the persistent CG solve (needed by the direct-implicit form, whose
    // operator is not separable; used for the explicit form too when it fits)
    const bool cg_ok = pcg_supported(c) != 0;
    c->use_pcg = c->implicit && cg_ok;
    if (c->implicit) {
        if (!cg_ok) return fail("implicit_es: the grid exceeds the CG Poisson solve (radial nodes a multiple of 4 and at most 16 per CTA of the cluster, at most 384 interior node rows, shared memory)");
        // Eq. facecharge uses the chi-free face coefficients: every face of a
        // turn node must see chi = 0, i.e. both nodes above the plasma rows
        for (int k = 0; k < N; ++k)
            for (int n : c->turn_nodes[k])
                if (n / NR <= c->i_win + 1) return fail("implicit_es: a turn node touches the plasma rows");
    }
    if (c->use_pcg) pcg_alloc(c, az, arp, arm, c->ps_mu);
    cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        set_error(std::string("CUDA error during init: ") + cudaGetErrorString(err));
        return PP_E_CUDA;
    }
    return PP_OK;
}

// ---------------------------------------------------------------- vacuum verification
// Z_vac of current sheets in vacuum (the paper's particle-free Tests 1-3,
// Sec. 3.1-3.3): the unit problems K U_k = g_k (Eq. unitfield, MQS) on the
// device with the FP64 separable solver, Dirichlet values on the boundary
// nodes (zero, or prescribed per unit problem), and the projection of
// Eq. zvac with eps_rec (Eq. reciprocity) on the host.
int vacuum_impedance(const pp_vacuum_problem* p, const double* boundary, double* zvac, double* eps_rec,
                     double* ufields) {
    if (p->nr < 3 || p->nz < 3 || p->r_max <= 0 || p->z_max <= 0 || p->freq <= 0)
        return fail("pp_vacuum_impedance: grid and frequency must be positive (nr, nz >= 3)");
    if (p->nr > 1024 || p->nz > 8192) return fail("pp_vacuum_impedance: grid too large (nr <= 1024, nz <= 8192)");
    const int N = p->n_src;
    if (N < 1 || N > PP_MAX_TURNS) return fail("pp_vacuum_impedance: n_src out of range");
    for (int k = 0; k < N; ++k)
        if (p->src_j[k] < 1 || p->src_j[k] > p->nr - 1 || p->src_i0[k] < 1 || p->src_i1[k] > p->nz - 1 ||
            p->src_i1[k] < p->src_i0[k])
            return fail("pp_vacuum_impedance: a sheet lies outside the interior nodes");
    Cell* c = new Cell();
    c->NR = p->nr + 1;
    c->NZ = p->nz + 1;
    c->nnodes = c->NR * c->NZ;
    c->dr = p->r_max / p->nr;
    c->dz = p->z_max / p->nz;
    c->omega = 2.0 * kPi * p->freq;
    c->eps_row.assign(p->nz, 1.0);
    build_helmholtz(c, 0.0);
    const int NR = c->NR, NZ = c->NZ, rows = c->hs.rows, MH = c->hs.M;
    const size_t nint = (size_t)rows * MH;
    const double dr = c->dr, dz = c->dz;
    int rc = PP_OK;
    if (!c->d_hstage) {
        set_error("pp_vacuum_impedance: cudaMalloc failed");
        rc = PP_E_CUDA;
    }
    std::vector<double> U((size_t)N * c->nnodes, 0.0), rhs(nint), sol(nint);
    std::vector<double> gval(N);
    for (int k = 0; k < N && rc == PP_OK; ++k) {
        gval[k] = 1.0 / ((p->src_i1[k] - p->src_i0[k] + 1) * dz * dr);
        const double* bnd = boundary ? boundary + (size_t)k * c->nnodes : nullptr;
        // right-hand side mu0 w g_k of the interior equations, less the
        // couplings to the boundary nodes' prescribed values
        for (int ii = 0; ii < rows; ++ii)
            for (int jj = 0; jj < MH; ++jj) {
                const int i = ii + 1, j = jj + 1;
                double v = 0.0;
                if (j == p->src_j[k] && i >= p->src_i0[k] && i <= p->src_i1[k]) v = kMu0 * c->omega * gval[k];
                if (bnd) {
                    const double R = j * dr;
                    if (i == 1) v -= bnd[j] / (dz * dz);
                    if (i == NZ - 2) v -= bnd[(size_t)(NZ - 1) * NR + j] / (dz * dz);
                    if (j == 1) v -= (R - dr / 2) / (R * dr * dr) * bnd[(size_t)i * NR];
                    if (j == NR - 2) v -= (R + dr / 2) / (R * dr * dr) * bnd[(size_t)i * NR + NR - 1];
                }
                rhs[(size_t)ii * MH + jj] = v;
            }
        cudaMemcpy(c->d_hstage, rhs.data(), sizeof(double) * nint, cudaMemcpyHostToDevice);
        sep_solve<double>(c->hs, c->d_hstage, c->d_hstage + nint, 0, nullptr);
        const cudaError_t e = cudaMemcpy(sol.data(), c->d_hstage + nint, sizeof(double) * nint, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error(std::string("pp_vacuum_impedance: ") + cudaGetErrorString(e));
            rc = PP_E_CUDA;
            break;
        }
        double* Uk = U.data() + (size_t)k * c->nnodes;
        for (int n = 0; n < c->nnodes; ++n) {
            const int i = n / NR, j = n % NR;
            if (i == 0 || i == NZ - 1 || j == 0 || j == NR - 1)
                Uk[n] = bnd ? bnd[n] : 0.0;
            else
                Uk[n] = sol[(size_t)(i - 1) * MH + (j - 1)];
        }
    }
    if (rc == PP_OK) {
        // Eq. zvac: Z_kl = -i sum_n g_k U_l 2 pi R dz dR over sheet k's nodes
        double zmax = 0.0, dmax = 0.0;
        for (int k = 0; k < N; ++k)
            for (int l = 0; l < N; ++l) {
                double s = 0.0;
                const int j = p->src_j[k];
                for (int i = p->src_i0[k]; i <= p->src_i1[k]; ++i)
                    s += gval[k] * U[(size_t)l * c->nnodes + (size_t)i * NR + j] * 2 * kPi * (j * dr) * dz * dr;
                zvac[2 * (k * N + l)] = 0.0;
                zvac[2 * (k * N + l) + 1] = -s;
            }
        for (int k = 0; k < N; ++k)
            for (int l = 0; l < N; ++l) {
                zmax = std::max(zmax, std::fabs(zvac[2 * (k * N + l) + 1]));
                dmax = std::max(dmax, std::fabs(zvac[2 * (k * N + l) + 1] - zvac[2 * (l * N + k) + 1]));
            }
        if (eps_rec) *eps_rec = zmax > 0 ? dmax / zmax : 0.0;
        if (ufields) memcpy(ufields, U.data(), sizeof(double) * U.size());
    }
    cudaDeviceSynchronize();
    for (void* q : c->allocs) cudaFree(q);
    delete c;
    return rc;
}

// Conductor charges of current-sheet conductors in a uniform dielectric (the
// electrostatic channel of the paper's Test 3, Sec. 3.3): for each unit
// problem l the sheets carry the potentials sheet_v[l][k], every boundary
// node its prescribed value (the axial rows and the outer radius; no R- face
// on the axis), and Laplace's equation (Eq. poisson without charge, the FV
// operator of Eq. epseff with eps_r uniform) holds on the free nodes.  The
// sheets span every interior node row, so with their columns as Dirichlet
// columns the operator stays separable: a radial generalised eigenbasis on
// the free columns and per-mode tridiagonal solves in z, in FP64 on the
// device.  C[k][l] is the Gauss-law charge of sheet k (Eq. facecharge over
// its external faces, Eq. areas) in unit problem l.
int vacuum_capacitance(const pp_vacuum_problem* p, double eps_r, const double* sheet_v, const double* boundary,
                       double* C, double* phis) {
    if (p->nr < 3 || p->nz < 3 || p->r_max <= 0 || p->z_max <= 0 || !(eps_r > 0))
        return fail("pp_vacuum_capacitance: grid and eps_r must be positive (nr, nz >= 3)");
    if (p->nr > 1024 || p->nz > 8192) return fail("pp_vacuum_capacitance: grid too large (nr <= 1024, nz <= 8192)");
    const int N = p->n_src;
    if (N < 1 || N > PP_MAX_TURNS) return fail("pp_vacuum_capacitance: n_src out of range");
    const int NR = p->nr + 1, NZ = p->nz + 1, rows = NZ - 2;
    std::vector<int> col_sheet(NR, -1);
    for (int k = 0; k < N; ++k) {
        if (p->src_j[k] < 1 || p->src_j[k] > p->nr - 1 || p->src_i0[k] != 1 || p->src_i1[k] != p->nz - 1)
            return fail("pp_vacuum_capacitance: every sheet must span all interior node rows of an interior column");
        if (col_sheet[p->src_j[k]] >= 0) return fail("pp_vacuum_capacitance: two sheets share a column");
        col_sheet[p->src_j[k]] = k;
    }
    const double dr = p->r_max / p->nr, dz = p->z_max / p->nz;
    // free columns: the axis and every column below the outer radius that is
    // not a sheet
    std::vector<int> F;
    for (int j = 0; j <= NR - 2; ++j)
        if (col_sheet[j] < 0) F.push_back(j);
    const int M = (int)F.size();
    auto area_z = [&](int j) { return j == 0 ? kPi * (dr / 2) * (dr / 2) : 2 * kPi * (j * dr) * dr; };
    auto rface = [&](int j, int s) { return 2 * kPi * (j * dr + s * dr / 2) * dz / dr; };   // A_r / dR
    // radial operator on the free columns (couplings to sheet columns and to
    // the outer radius go to the right-hand side) and the z-face weights
    std::vector<double> T((size_t)M * M, 0.0), D(M);
    for (int a = 0; a < M; ++a) {
        const int j = F[a];
        double diag = 0.0;
        for (int s = -1; s <= 1; s += 2) {
            if (j == 0 && s < 0) continue;
            const double c = rface(j, s);
            diag -= c;
            const int jn = j + s;
            if (jn >= 0 && jn <= NR - 2 && col_sheet[jn] < 0) {
                const int b = (int)(std::lower_bound(F.begin(), F.end(), jn) - F.begin());
                T[(size_t)a * M + b] = c;
            }
        }
        T[(size_t)a * M + a] = diag;
        D[a] = area_z(j) / dz;
    }
    std::vector<double> mu, V;
    radial_basis(T, D, M, mu, V);
    // D d2z phi + T phi = rhs with T V = D V Lambda, V' D V = I: per mode
    // d2z c + Lambda c = V' rhs (forward transform V', backward V)
    std::vector<double> Vf((size_t)M * M), Vb((size_t)M * M);
    for (int a = 0; a < M; ++a)
        for (int m = 0; m < M; ++m) {
            Vf[(size_t)a * M + m] = V[(size_t)a * M + m];
            Vb[(size_t)m * M + a] = V[(size_t)a * M + m];
        }
    std::vector<double> lo(rows), up(rows), diag((size_t)rows * M), cp, invd;
    for (int ii = 0; ii < rows; ++ii) {
        lo[ii] = ii > 0 ? 1.0 : 0.0;
        up[ii] = 1.0;
        for (int m = 0; m < M; ++m) diag[(size_t)ii * M + m] = -2.0 + mu[m];
    }
    thomas_factors(lo, up, diag, rows, M, cp, invd);
    Cell* c = new Cell();
    SepSolver<double>& s = c->hs;
    s.rows = rows;
    s.M = M;
    s.Vf = upload<double>(c, Vf);
    s.Vb = upload<double>(c, Vb);
    s.cp = upload<double>(c, cp);
    s.invd = upload<double>(c, invd);
    s.lo = upload<double>(c, lo);
    s.t0 = c->alloc<double>((size_t)rows * M);
    s.t1 = c->alloc<double>((size_t)rows * M);
    double* stage = c->alloc<double>((size_t)2 * rows * M);
    int rc = PP_OK;
    if (!stage || !s.t1) {
        set_error("pp_vacuum_capacitance: cudaMalloc failed");
        rc = PP_E_CUDA;
    }
    const size_t nint = (size_t)rows * M, nn = (size_t)NR * NZ;
    std::vector<double> rhs(nint), sol(nint), phi(nn);
    for (int l = 0; l < N && rc == PP_OK; ++l) {
        const double* bnd = boundary + (size_t)l * nn;
        const double* vk = sheet_v + (size_t)l * N;
        // the node potentials known before the solve
        for (size_t n = 0; n < nn; ++n) {
            const int i = (int)(n / NR), j = (int)(n % NR);
            const bool edge = i == 0 || i == NZ - 1 || j == NR - 1;
            phi[n] = edge ? bnd[n] : (col_sheet[j] >= 0 ? vk[col_sheet[j]] : 0.0);
        }
        // right-hand side of the free nodes' equations (divided by eps):
        // minus the couplings to the known potentials
        for (int ii = 0; ii < rows; ++ii) {
            const int i = ii + 1;
            for (int a = 0; a < M; ++a) {
                const int j = F[a];
                double v = 0.0;
                if (i == 1) v -= D[a] * phi[(size_t)j];
                if (i == NZ - 2) v -= D[a] * phi[(size_t)(NZ - 1) * NR + j];
                for (int sg = -1; sg <= 1; sg += 2) {
                    if (j == 0 && sg < 0) continue;
                    const int jn = j + sg;
                    if (jn == NR - 1 || col_sheet[jn] >= 0) v -= rface(j, sg) * phi[(size_t)i * NR + jn];
                }
                rhs[(size_t)ii * M + a] = v;
            }
        }
        cudaMemcpy(stage, rhs.data(), sizeof(double) * nint, cudaMemcpyHostToDevice);
        sep_solve<double>(s, stage, stage + nint, 0, nullptr);
        const cudaError_t e = cudaMemcpy(sol.data(), stage + nint, sizeof(double) * nint, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error(std::string("pp_vacuum_capacitance: ") + cudaGetErrorString(e));
            rc = PP_E_CUDA;
            break;
        }
        for (int ii = 0; ii < rows; ++ii)
            for (int a = 0; a < M; ++a) phi[(size_t)(ii + 1) * NR + F[a]] = sol[(size_t)ii * M + a];
        if (phis) memcpy(phis + (size_t)l * nn, phi.data(), sizeof(double) * nn);
        // Eq. facecharge: each sheet node's faces to nodes that are not of
        // the same sheet (its vertical neighbours are, except at the ends)
        for (int k = 0; k < N; ++k) {
            const int j = p->src_j[k];
            double q = 0.0;
            for (int i = 1; i <= NZ - 2; ++i) {
                const double pc = phi[(size_t)i * NR + j];
                if (i == 1) q += area_z(j) / dz * (pc - phi[(size_t)j]);
                if (i == NZ - 2) q += area_z(j) / dz * (pc - phi[(size_t)(NZ - 1) * NR + j]);
                q += rface(j, +1) * (pc - phi[(size_t)i * NR + j + 1]);
                q += rface(j, -1) * (pc - phi[(size_t)i * NR + j - 1]);
            }
            C[(size_t)k * N + l] = kEps0 * eps_r * q;
        }
    }
    cudaDeviceSynchronize();
    for (void* q : c->allocs) cudaFree(q);
    delete c;
    return rc;
}

}  // namespace pp
