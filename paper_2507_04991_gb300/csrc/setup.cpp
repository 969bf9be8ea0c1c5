// Host-side setup of a P-ERRK context: LGL tables, metric terms, mesh and
// tableau validation, partition-major element ordering, work chunks and the
// per-stage coefficient tables.  Plain C++ (no CUDA).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "perrk_internal.h"

namespace perrk {

// LGL nodes/weights for N = 3 from their closed forms (roots of P_3' are
// +-1/sqrt(5); weights 2 / (N (N+1) P_N(x)^2)) and the differentiation matrix
// D_ij = l_j'(x_i) from barycentric weights, in long double.
void lgl_tables(std::vector<double> &x, std::vector<double> &w, std::vector<double> &D) {
    const long double s5 = 1.0L / std::sqrt(5.0L);
    long double xl[4] = {-1.0L, -s5, s5, 1.0L};
    x.assign(4, 0.0);
    w.assign(4, 0.0);
    D.assign(16, 0.0);
    for (int i = 0; i < 4; ++i) {
        x[i] = (double)xl[i];
        long double P3 = 0.5L * (5.0L * xl[i] * xl[i] * xl[i] - 3.0L * xl[i]);
        w[i] = (double)(2.0L / (12.0L * P3 * P3));
    }
    long double lam[4];
    for (int j = 0; j < 4; ++j) {
        lam[j] = 1.0L;
        for (int k = 0; k < 4; ++k)
            if (k != j) lam[j] /= (xl[j] - xl[k]);
    }
    for (int i = 0; i < 4; ++i) {
        long double diag = 0.0L;
        for (int j = 0; j < 4; ++j) {
            if (i == j) continue;
            long double v = (lam[j] / lam[i]) / (xl[i] - xl[j]);
            D[i * 4 + j] = (double)v;
            diag -= v;
        }
        D[i * 4 + i] = (double)diag;
    }
}

namespace {

int min_E(int p) { return p == 2 ? 2 : (p == 3 ? 3 : 5); }

int node_index(int dim, int i, int j, int k) { return i + 4 * j + (dim == 3 ? 16 * k : 0); }

// Face node kk of face f: node index inside the element.
int face_node(int dim, int f, int kk) {
    int k = f / 2, s = f % 2, e = s ? 3 : 0;
    if (dim == 1) return e;
    if (dim == 2) return k == 0 ? e + 4 * kk : kk + 4 * e;
    int a = kk % 4, b = kk / 4;
    if (k == 0) return e + 4 * a + 16 * b;
    if (k == 1) return a + 4 * e + 16 * b;
    return a + 4 * b + 16 * e;
}

struct ElemGeo {
    // derivative of coordinate comp along reference direction k at each node
    double dx[3][3][64];
};

void elem_derivatives(int dim, const double *xe, const std::vector<double> &D, ElemGeo &g) {
    const int NP = ipow4(dim);
    for (int k = 0; k < dim; ++k)
        for (int comp = 0; comp < dim; ++comp)
            for (int q = 0; q < NP; ++q) {
                int idx[3] = {q % 4, (q / 4) % 4, q / 16};
                double acc = 0.0;
                for (int m = 0; m < 4; ++m) {
                    int id2[3] = {idx[0], idx[1], idx[2]};
                    id2[k] = m;
                    acc += D[idx[k] * 4 + m] * xe[node_index(dim, id2[0], id2[1], id2[2]) * dim + comp];
                }
                g.dx[k][comp][q] = acc;
            }
}

}  // namespace

// Lagrange basis of the LGL nodes x at the point s (extended precision).
static void lagrange_at(const std::vector<double> &x, long double s, long double *l) {
    const int n = (int)x.size();
    for (int j = 0; j < n; ++j) {
        long double v = 1.0L;
        for (int k = 0; k < n; ++k)
            if (k != j) v *= (s - (long double)x[k]) / ((long double)x[j] - (long double)x[k]);
        l[j] = v;
    }
}

// Operators of the L2 projection mortars (N = 3): P_m[j][i] = l_i((x_j -+ 1)/2)
// and R_m = M^-1 P_m^T M with the exact mass matrix M_ij = int l_i l_j
// (four-point Gauss-Legendre, exact for degree 7), index (m 4 + j) 4 + i.
void mortar_operators(const std::vector<double> &x, double *P, double *R) {
    const long double r = sqrtl(6.0L / 5.0L);
    const long double gx[4] = {-sqrtl(3.0L / 7.0L + 2.0L / 7.0L * r), -sqrtl(3.0L / 7.0L - 2.0L / 7.0L * r),
                               sqrtl(3.0L / 7.0L - 2.0L / 7.0L * r), sqrtl(3.0L / 7.0L + 2.0L / 7.0L * r)};
    const long double s30 = sqrtl(30.0L);
    const long double gw[4] = {(18.0L - s30) / 36.0L, (18.0L + s30) / 36.0L, (18.0L + s30) / 36.0L,
                               (18.0L - s30) / 36.0L};
    long double M[4][4] = {}, l[4];
    for (int g = 0; g < 4; ++g) {
        lagrange_at(x, gx[g], l);
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) M[i][j] += gw[g] * l[i] * l[j];
    }
    // M^-1 by Gauss-Jordan elimination (M is symmetric positive definite)
    long double A[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) A[i][j] = j < 4 ? M[i][j] : (j - 4 == i ? 1.0L : 0.0L);
    for (int c = 0; c < 4; ++c) {
        const long double piv = A[c][c];
        for (int j = 0; j < 8; ++j) A[c][j] /= piv;
        for (int i = 0; i < 4; ++i)
            if (i != c) {
                const long double f = A[i][c];
                for (int j = 0; j < 8; ++j) A[i][j] -= f * A[c][j];
            }
    }
    for (int m = 0; m < 2; ++m) {
        long double Pm[4][4];
        for (int j = 0; j < 4; ++j) {
            lagrange_at(x, 0.5L * ((long double)x[j] + (m ? 1.0L : -1.0L)), l);
            for (int i = 0; i < 4; ++i) Pm[j][i] = l[i];
        }
        long double PtM[4][4] = {};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                for (int k = 0; k < 4; ++k) PtM[i][j] += Pm[k][i] * M[k][j];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                long double v = 0.0L;
                for (int k = 0; k < 4; ++k) v += A[i][4 + k] * PtM[k][j];
                R[(m * 4 + i) * 4 + j] = (double)v;
                P[(m * 4 + i) * 4 + j] = (double)Pm[i][j];
            }
    }
}


perrk_status build_ctx(Ctx &c, int n, const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme,
                       const perrk_options *opts, std::string &err) {
    char buf[256];
    auto fail = [&](const char *m) {
        err = m;
        return PERRK_INVALID_ARG;
    };
    if (n < 1 || !mesh || !scheme || !opts) return fail("null argument or n < 1");
    const perrk_scheme_desc &s0 = scheme[0];
    int dim = mesh[0].dim;
    int eq = s0.equation;
    int eq_dim = eq == PERRK_BURGERS_1D ? 1 : (eq == PERRK_EULER_1D ? 1 : (eq == PERRK_EULER_2D ? 2 : (eq == PERRK_EULER_3D ? 3 : 0)));
    if (eq_dim == 0) return fail("unknown equation");
    if (dim != eq_dim) return fail("mesh dim does not match the equation");
    if (s0.surface_flux != PERRK_SURFACE_EC && s0.surface_flux != PERRK_SURFACE_ES_RUSANOV) return fail("unknown surface flux");
    if (s0.volume_flux != PERRK_VOLUME_EC) return fail("unknown volume flux");
    if (eq != PERRK_BURGERS_1D && !(s0.gamma_gas > 1.0)) return fail("gamma_gas must be > 1");
    if (!(s0.mu >= 0.0) || !std::isfinite(s0.mu)) return fail("mu must be finite and >= 0");
    if (s0.mu > 0.0) {
        if (eq != PERRK_EULER_2D && eq != PERRK_EULER_3D) return fail("viscous terms need the 2D or 3D Euler equations");
        if (!(s0.prandtl > 0.0) || !std::isfinite(s0.prandtl)) return fail("prandtl must be finite and > 0");
    }
    if (opts->precision != PERRK_FP64 && opts->precision != PERRK_MIXED) return fail("unknown precision");
    if (opts->newton_max_it < 0 || opts->newton_max_it > 64) return fail("newton_max_it out of range [0, 64]");
    if (!(opts->newton_tol_r >= 0.0) || !(opts->newton_tol_g >= 0.0)) return fail("negative Newton tolerance");
    if (opts->guess < 0 || opts->guess > 2 || opts->target < 0 || opts->target > 2) return fail("bad guess/target enum");
    if (opts->solver < 0 || opts->solver > 2) return fail("unknown relaxation solver");
    if (opts->solver != PERRK_SOLVER_NEWTON &&
        !(std::isfinite(opts->bracket_lo) && std::isfinite(opts->bracket_hi) && opts->bracket_lo < opts->bracket_hi))
        return fail("bisection / secant need finite bracket_lo < bracket_hi");

    c.dim = dim;
    c.NP = ipow4(dim);
    c.V = eq == PERRK_BURGERS_1D ? 1 : dim + 2;
    c.equation = eq;
    c.surface = s0.surface_flux;
    c.gamma_gas = eq == PERRK_BURGERS_1D ? 1.4 : s0.gamma_gas;
    c.viscous = s0.mu > 0.0;
    c.mu = s0.mu;
    c.prandtl = c.viscous ? s0.prandtl : 0.75;
    c.opt = *opts;
    c.p = s0.order;
    c.n_inst = n;
    std::vector<double> x;
    lgl_tables(x, c.lgl_w, c.lgl_D);

    // ---------------------------------------------------------- instances
    c.inst.assign(n, Instance());
    int S = 0, elem0 = 0, gp0 = 0;
    for (int k = 0; k < n; ++k) {
        const perrk_mesh_desc &m = mesh[k];
        const perrk_scheme_desc &sc = scheme[k];
        if (m.dim != dim || sc.equation != eq || sc.surface_flux != s0.surface_flux || sc.order != s0.order ||
            sc.gamma_gas != s0.gamma_gas || sc.mu != s0.mu || (s0.mu > 0.0 && sc.prandtl != s0.prandtl))
            return fail("instances must share dim, equation, fluxes, gamma_gas, viscosity and order");
        if (m.N != 3) return fail("only N = 3 is supported");
        if (m.n_elem <= 0 || !m.node_coords || !m.faces || !m.partition_id) return fail("empty mesh or null arrays");
        if (m.n_mortars < 0 || (m.n_mortars > 0 && !m.mortars)) return fail("n_mortars < 0 or null mortar rows");
        if (m.n_mortars == 0 && m.n_faces != m.n_elem * dim) return fail("n_faces must equal n_elem * dim");
        if (m.n_mortars > 0 && dim != 2) return fail("mortars (non-conforming faces) are supported in 2D only");
        if (m.n_faces < 0) return fail("n_faces < 0");
        if (sc.order < 2 || sc.order > 4) return fail("order must be 2, 3 or 4");
        if (sc.R < 1 || sc.R > kMaxR) return fail("R out of range");
        if (sc.S < 2 || sc.S > 64) return fail("S out of range [2, 64]");
        if (!sc.E || !sc.c || !sc.b || !sc.a1 || !sc.asub) return fail("null tableau arrays");
        Instance &I = c.inst[k];
        I.elem0 = elem0;
        I.n_elem = m.n_elem;
        I.gp0 = gp0;
        I.R = sc.R;
        I.S = sc.S;
        I.p = sc.order;
        I.E.assign(sc.E, sc.E + sc.R);
        I.c.assign(sc.c, sc.c + sc.S);
        I.b.assign(sc.b, sc.b + sc.S);
        I.a1.assign(sc.a1, sc.a1 + sc.R * sc.S);
        I.asub.assign(sc.asub, sc.asub + sc.R * sc.S);
        // tableau checks (eq. InternalConsistency, eq. Conservation, activity pattern)
        int Emin = 1 << 30;
        for (int r = 0; r < sc.R; ++r) {
            int E = sc.E[r];
            if (E < min_E(sc.order) || E > sc.S) {
                snprintf(buf, sizeof buf, "instance %d: E[%d] = %d outside [%d, S = %d]", k, r, E, min_E(sc.order), sc.S);
                err = buf;
                return PERRK_INVALID_ARG;
            }
            Emin = std::min(Emin, E);
            for (int i = 0; i < sc.S; ++i) {
                double a1 = sc.a1[r * sc.S + i], as = sc.asub[r * sc.S + i], ci = sc.c[i];
                if (!std::isfinite(a1) || !std::isfinite(as)) return fail("non-finite tableau entry");
                if (i == 0) {
                    if (a1 != 0.0 || as != 0.0 || ci != 0.0) return fail("stage 1 row must be zero with c_1 = 0");
                    continue;
                }
                if (std::fabs(a1 + as - ci) > 1e-12 * (1.0 + std::fabs(ci)))
                    return fail("row sum a1 + asub differs from c_i (internal consistency)");
                int stage = i + 1;  // 1-based
                bool active = stage >= sc.S - E + 2;
                bool first = stage == sc.S - E + 2;
                if (!active && (as != 0.0)) return fail("inactive row with nonzero K_{i-1} coefficient");
                if (first && stage >= 3 && as != 0.0) return fail("first active row must not use K_{i-1}");
            }
        }
        for (int i = 0; i < sc.S; ++i) {
            if (!std::isfinite(sc.b[i])) return fail("non-finite b");
            int stage = i + 1;
            if (sc.b[i] != 0.0 && !(stage == 1 || stage >= sc.S - Emin + 2))
                return fail("b_i != 0 at a stage where some member is inactive");
        }
        for (int e = 0; e < m.n_elem; ++e)
            if (m.partition_id[e] < 0 || m.partition_id[e] >= sc.R) return fail("partition id out of range");
        S = std::max(S, sc.S);
        elem0 += m.n_elem;
        gp0 += sc.R;
    }
    c.S = S;
    c.n_elem = elem0;
    c.n_gp = gp0;

    // ---------------------------------------------------------- geometry
    const int NP = c.NP, NF = 2 * dim, NFP = ipow4(dim - 1);
    const size_t NE = (size_t)c.n_elem;
    c.gp_of_elem.assign(NE, 0);
    c.E_of_gp.assign(c.n_gp, 0);
    c.nbr.assign(NE * NF, -1);
    c.wJ.assign(NE * NP, 0.0);
    std::vector<double> Ja(NE * NP * 9, 0.0), J(NE * NP, 0.0);
    // box detection: every element an axis-aligned box with LGL node placement
    bool all_box = true;
    for (int k = 0; k < n; ++k) {
        const perrk_mesh_desc &m = mesh[k];
        const Instance &I = c.inst[k];
        for (int r = 0; r < I.R; ++r) c.E_of_gp[I.gp0 + r] = I.E[r];
        for (int e = 0; e < m.n_elem; ++e) {
            size_t ge = (size_t)I.elem0 + e;
            c.gp_of_elem[ge] = I.gp0 + m.partition_id[e];
            const double *xe = m.node_coords + (size_t)e * NP * dim;
            for (int q = 0; q < NP * dim; ++q)
                if (!std::isfinite(xe[q])) return fail("non-finite node coordinate");
            ElemGeo g;
            elem_derivatives(dim, xe, c.lgl_D, g);
            // affine-box tolerance: D x carries cancellation error ~ eps sum|D||x|
            double scale = 0.0, xmax = 0.0;
            for (int q = 0; q < NP; ++q)
                for (int a = 0; a < dim; ++a) {
                    xmax = std::max(xmax, std::fabs(xe[q * dim + a]));
                    for (int b = 0; b < dim; ++b) scale = std::max(scale, std::fabs(g.dx[a][b][q]));
                }
            const double box_tol = 1e-12 * (scale + xmax);
            for (int q = 0; q < NP; ++q) {
                double *ja = &Ja[(ge * NP + q) * 9];
                double Jq;
                if (dim == 1) {
                    Jq = g.dx[0][0][q];
                    ja[0] = 1.0;
                } else if (dim == 2) {
                    double xx = g.dx[0][0][q], xy = g.dx[1][0][q], yx = g.dx[0][1][q], yy = g.dx[1][1][q];
                    Jq = xx * yy - xy * yx;
                    ja[0] = yy;   // Ja^1 = (y_eta, -x_eta)
                    ja[1] = -xy;
                    ja[3] = -yx;  // Ja^2 = (-y_xi, x_xi)
                    ja[4] = xx;
                } else {
                    // cross-product form Ja^1 = x_eta x x_zeta, Ja^2 = x_zeta x x_xi, Ja^3 = x_xi x x_eta
                    double a[3], b[3], cc[3];
                    for (int t = 0; t < 3; ++t) {
                        a[t] = g.dx[0][t][q];
                        b[t] = g.dx[1][t][q];
                        cc[t] = g.dx[2][t][q];
                    }
                    auto cross = [](const double *u, const double *v, double *o) {
                        o[0] = u[1] * v[2] - u[2] * v[1];
                        o[1] = u[2] * v[0] - u[0] * v[2];
                        o[2] = u[0] * v[1] - u[1] * v[0];
                    };
                    cross(b, cc, ja);
                    cross(cc, a, ja + 3);
                    cross(a, b, ja + 6);
                    Jq = a[0] * ja[0] + a[1] * ja[1] + a[2] * ja[2];
                }
                if (!(Jq > 0.0)) {
                    snprintf(buf, sizeof buf, "instance %d element %d: non-positive Jacobian", k, e);
                    err = buf;
                    return PERRK_INVALID_ARG;
                }
                J[ge * NP + q] = Jq;
                // off-diagonal derivative terms vanish for axis-aligned boxes
                for (int a = 0; a < dim; ++a)
                    for (int b = 0; b < dim; ++b)
                        if (a != b && std::fabs(g.dx[a][b][q]) > box_tol) all_box = false;
            }
            if (dim >= 2) {
                // and the diagonal derivatives are constant over the element
                for (int a = 0; a < dim; ++a)
                    for (int q = 1; q < NP; ++q)
                        if (std::fabs(g.dx[a][a][q] - g.dx[a][a][0]) > box_tol) all_box = false;
            } else {
                for (int q = 1; q < NP; ++q)
                    if (std::fabs(g.dx[0][0][q] - g.dx[0][0][0]) > box_tol) all_box = false;
            }
            for (int q = 0; q < NP; ++q) {
                int idx[3] = {q % 4, (q / 4) % 4, q / 16};
                double wq = 1.0;
                for (int a = 0; a < dim; ++a) wq *= c.lgl_w[idx[a]];
                c.wJ[ge * NP + q] = wq * J[ge * NP + q];
            }
        }
    }
    if (dim == 3 && !all_box) return fail("3D elements must be axis-aligned boxes (cross-product metrics)");
    if (dim == 1 && !all_box) return fail("1D elements must be affine (LGL nodes equally mapped)");
    c.curved = !all_box;

    // ---------------------------------------------------------- faces
    for (int k = 0; k < n; ++k) {
        const perrk_mesh_desc &m = mesh[k];
        const Instance &I = c.inst[k];
        std::vector<int> seen((size_t)m.n_elem * NF, 0);
        for (int fi = 0; fi < m.n_faces; ++fi) {
            const int32_t *row = m.faces + 4 * fi;
            int eL = row[0], fL = row[1], eR = row[2], fR = row[3];
            if (eL < 0 || eL >= m.n_elem || eR < 0 || eR >= m.n_elem) return fail("face element index out of range");
            if (fL < 0 || fL >= NF || (fL % 2) != 1 || fR != fL - 1) return fail("face row must pair '+' face fL with fR = fL - 1");
            if (seen[(size_t)eL * NF + fL]++ || seen[(size_t)eR * NF + fR]++) return fail("element face used twice");
            // translation check: face nodes coincide up to a constant shift (periodic pairs)
            const double *xl = m.node_coords + (size_t)eL * NP * dim;
            const double *xr = m.node_coords + (size_t)eR * NP * dim;
            double sh[3] = {0, 0, 0}, sc2 = 0.0;
            for (int kk = 0; kk < NFP; ++kk) {
                int ql = face_node(dim, fL, kk), qr = face_node(dim, fR, kk);
                for (int a = 0; a < dim; ++a) {
                    double dd = xl[ql * dim + a] - xr[qr * dim + a];
                    if (kk == 0) sh[a] = dd;
                    sc2 = std::max(sc2, std::fabs(xl[ql * dim + a]) + std::fabs(xr[qr * dim + a]));
                    if (std::fabs(dd - sh[a]) > 1e-9 * (1.0 + sc2)) return fail("face nodes do not match (orientation or geometry)");
                }
            }
            size_t gL = (size_t)I.elem0 + eL, gR = (size_t)I.elem0 + eR;
            c.nbr[gL * NF + fL] = (int32_t)gR;
            c.nbr[gR * NF + fR] = (int32_t)gL;
        }
    }
    // ---------------------------------------------------------- mortars
    c.mortars.clear();
    for (int k = 0; k < n; ++k) {
        const perrk_mesh_desc &m = mesh[k];
        if (m.n_mortars == 0) continue;
        const Instance &I = c.inst[k];
        if (!all_box) return fail("mortars need axis-aligned box elements");
        if (c.viscous) return fail("viscous terms on non-conforming meshes are not supported");
        std::vector<int> seen((size_t)m.n_elem * NF, 0);
        for (int fi = 0; fi < m.n_faces; ++fi) {
            const int32_t *row = m.faces + 4 * fi;
            seen[(size_t)row[0] * NF + row[1]]++;
            seen[(size_t)row[2] * NF + row[3]]++;
        }
        for (int mi = 0; mi < m.n_mortars; ++mi) {
            const int32_t *row = m.mortars + 4 * mi;
            const int ec = row[0], fc = row[1], el = row[2], eh = row[3];
            if (ec < 0 || ec >= m.n_elem || el < 0 || el >= m.n_elem || eh < 0 || eh >= m.n_elem || fc < 0 ||
                fc >= NF || el == eh || el == ec || eh == ec)
                return fail("mortar row out of range");
            const int ff = fc ^ 1;
            if (seen[(size_t)ec * NF + fc]++ || seen[(size_t)el * NF + ff]++ || seen[(size_t)eh * NF + ff]++)
                return fail("element face used twice");
            // geometry: the fine faces are the two halves of the coarse face (up
            // to a common translation for periodic pairs), in tangential order
            const double *xc = m.node_coords + (size_t)ec * NP * dim;
            const int qc0 = face_node(dim, fc, 0), qc3 = face_node(dim, fc, NFP - 1);
            double sh[2] = {0, 0};
            bool first = true;
            for (int half = 0; half < 2; ++half) {
                const double *xf = m.node_coords + (size_t)(half ? eh : el) * NP * dim;
                for (int kk = 0; kk < NFP; ++kk) {
                    const double sloc = 0.5 * (x[kk] + (half ? 1.0 : -1.0));   // coarse face coordinate
                    const int qf = face_node(dim, ff, kk);
                    for (int a = 0; a < dim; ++a) {
                        const double want = 0.5 * (1.0 - sloc) * xc[qc0 * dim + a] + 0.5 * (1.0 + sloc) * xc[qc3 * dim + a];
                        const double dd = xf[qf * dim + a] - want;
                        if (first) sh[a] = dd;
                        const double scl = 1.0 + std::fabs(want) + std::fabs(xf[qf * dim + a]);
                        if (std::fabs(dd - sh[a]) > 1e-9 * scl) return fail("mortar faces are not the halves of the coarse face");
                    }
                    first = false;
                }
            }
            const int32_t g[4] = {(int32_t)(I.elem0 + ec), fc, (int32_t)(I.elem0 + el), (int32_t)(I.elem0 + eh)};
            c.mortars.insert(c.mortars.end(), g, g + 4);
            c.nbr[(size_t)g[0] * NF + fc] = g[0];   // no conforming partner: the stage kernels read the trace
            c.nbr[(size_t)g[2] * NF + ff] = g[2];
            c.nbr[(size_t)g[3] * NF + ff] = g[3];
        }
    }
    c.n_mortars = (int)(c.mortars.size() / 4);
    if (c.n_mortars > 0) mortar_operators(x, c.mortar_P, c.mortar_R);

    // every face of every element needs a partner (interior or periodic): the
    // method has no boundary conditions here, and the kernels index nbr[] directly
    for (size_t i = 0; i < c.nbr.size(); ++i)
        if (c.nbr[i] < 0) {
            snprintf(buf, sizeof buf, "element %zu face %zu has no partner face (boundary faces are not supported)",
                     i / (size_t)NF, i % (size_t)NF);
            err = buf;
            return PERRK_INVALID_ARG;
        }
    // canonical face normals: the '+' side's Ja^k at its face nodes, shared by both sides
    if (c.curved) {
        c.fnorm.assign(NE * NF * NFP * 2, 0.0);
        c.geo_node.assign(6 * NE * NP, 0.0);
        for (size_t e = 0; e < NE; ++e)
            for (int q = 0; q < NP; ++q) {
                const double *ja = &Ja[(e * NP + q) * 9];
                c.geo_node[0 * NE * NP + e * NP + q] = ja[0];
                c.geo_node[1 * NE * NP + e * NP + q] = ja[1];
                c.geo_node[2 * NE * NP + e * NP + q] = ja[3];
                c.geo_node[3 * NE * NP + e * NP + q] = ja[4];
                c.geo_node[4 * NE * NP + e * NP + q] = 1.0 / J[e * NP + q];
                c.geo_node[5 * NE * NP + e * NP + q] = c.wJ[e * NP + q];
            }
        for (size_t e = 0; e < NE; ++e)
            for (int f = 1; f < NF; f += 2) {
                size_t nb = (size_t)c.nbr[e * NF + f];
                int kdir = f / 2;
                for (int kk = 0; kk < NFP; ++kk) {
                    int q = face_node(dim, f, kk);
                    const double *ja = &Ja[(e * NP + q) * 9 + 3 * kdir];
                    for (int a = 0; a < 2; ++a) {
                        c.fnorm[((e * NF + f) * NFP + kk) * 2 + a] = ja[a];
                        c.fnorm[((nb * NF + (f - 1)) * NFP + kk) * 2 + a] = ja[a];
                    }
                }
            }
    } else {
        c.fnorm.assign(NE * NF, 0.0);
        c.geo_elem.assign(NE * 8, 0.0);
        for (size_t e = 0; e < NE; ++e) {
            for (int a = 0; a < dim; ++a) c.geo_elem[e * 8 + a] = Ja[(e * NP) * 9 + 3 * a + a];
            c.geo_elem[e * 8 + 3] = 1.0 / J[e * NP];
            c.geo_elem[e * 8 + 4] = J[e * NP];
        }
        for (size_t e = 0; e < NE; ++e)
            for (int f = 1; f < NF; f += 2) {
                size_t nb = (size_t)c.nbr[e * NF + f];
                double v = c.geo_elem[e * 8 + f / 2];
                c.fnorm[e * NF + f] = v;
                c.fnorm[nb * NF + (f - 1)] = v;
            }
        // a mortar face has no conforming partner: its normal is the element's own
        for (int mi = 0; mi < c.n_mortars; ++mi) {
            const int32_t *r = &c.mortars[4 * mi];
            const int fc = r[1];
            c.fnorm[(size_t)r[0] * NF + fc] = c.geo_elem[(size_t)r[0] * 8 + fc / 2];
            for (int h : {2, 3}) c.fnorm[(size_t)r[h] * NF + (fc ^ 1)] = c.geo_elem[(size_t)r[h] * 8 + fc / 2];
        }
    }

    // ---------------------------------------------------------- ordering
    // Partition-major (E descending), so that every stage's active elements
    // form a prefix.  Within a partition, instance by instance: in 3D along a
    // Morton (Z-order) curve of the element centroids, so that the elements
    // that concurrently running CTAs take form a compact block and the face
    // neighbours in every direction are near in processing order (L2 hits);
    // in 1D and 2D in the given order (on row-numbered meshes a neighbour is
    // at most one row away, and Morton order measured slower there).
    std::vector<uint64_t> zkey(NE, 0);
    for (int k = 0; k < n && dim == 3; ++k) {
        const perrk_mesh_desc &m = mesh[k];
        const Instance &I = c.inst[k];
        std::vector<double> cen((size_t)m.n_elem * dim, 0.0);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int e = 0; e < m.n_elem; ++e)
            for (int a = 0; a < dim; ++a) {
                double sum = 0.0;
                for (int q = 0; q < NP; ++q) sum += m.node_coords[((size_t)e * NP + q) * dim + a];
                const double v = sum / NP;
                cen[(size_t)e * dim + a] = v;
                lo[a] = std::min(lo[a], v);
                hi[a] = std::max(hi[a], v);
            }
        for (int e = 0; e < m.n_elem; ++e) {
            uint64_t code = 0;
            for (int a = 0; a < dim; ++a) {
                const double w = hi[a] - lo[a];
                const double t = w > 0.0 ? (cen[(size_t)e * dim + a] - lo[a]) / w : 0.0;
                const uint64_t qa = (uint64_t)std::min(65535.0, std::max(0.0, std::floor(t * 65535.0 + 0.5)));
                for (int bit = 0; bit < 16; ++bit) code |= ((qa >> bit) & 1u) << (bit * dim + a);
            }
            zkey[(size_t)I.elem0 + e] = code;
        }
    }
    std::vector<int32_t> inst_of(NE, 0);
    for (int k = 0; k < n; ++k)
        for (int e = 0; e < c.inst[k].n_elem; ++e) inst_of[(size_t)c.inst[k].elem0 + e] = k;
    c.elist.resize(NE);
    std::iota(c.elist.begin(), c.elist.end(), 0);
    std::stable_sort(c.elist.begin(), c.elist.end(), [&](int a, int b) {
        const int Ea = c.E_of_gp[c.gp_of_elem[a]], Eb = c.E_of_gp[c.gp_of_elem[b]];
        if (Ea != Eb) return Ea > Eb;
        if (inst_of[a] != inst_of[b]) return inst_of[a] < inst_of[b];
        return zkey[a] < zkey[b];
    });
    c.n_active.assign(S, 0);
    for (int i = 1; i <= S; ++i) {
        int cnt = 0;
        for (size_t e = 0; e < NE; ++e) {
            int E = c.E_of_gp[c.gp_of_elem[e]];
            if (i == 1 || i >= S - E + 2) ++cnt;
        }
        c.n_active[i - 1] = cnt;
    }
    // mortars: sorted by the largest E of their elements, so that the mortars
    // touching an active element form a prefix at every stage
    c.face_mortar.assign(NE * NF, -1);
    c.mortar_active.assign(S, 0);
    if (c.n_mortars > 0) {
        auto maxE = [&](int mi) {
            int E = 0;
            for (int j : {0, 2, 3}) E = std::max(E, c.E_of_gp[c.gp_of_elem[c.mortars[4 * mi + j]]]);
            return E;
        };
        std::vector<int> ord(c.n_mortars);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return maxE(a) > maxE(b); });
        std::vector<int32_t> sorted(c.mortars.size());
        for (int i = 0; i < c.n_mortars; ++i)
            for (int j = 0; j < 4; ++j) sorted[4 * i + j] = c.mortars[4 * ord[i] + j];
        c.mortars.swap(sorted);
        for (int mi = 0; mi < c.n_mortars; ++mi) {
            const int32_t *r = &c.mortars[4 * mi];
            c.face_mortar[(size_t)r[0] * NF + r[1]] = 3 * mi;
            c.face_mortar[(size_t)r[2] * NF + (r[1] ^ 1)] = 3 * mi + 1;
            c.face_mortar[(size_t)r[3] * NF + (r[1] ^ 1)] = 3 * mi + 2;
        }
        for (int i = 1; i <= S; ++i) {
            int cnt = 0;
            for (int mi = 0; mi < c.n_mortars; ++mi) {
                const int E = maxE(mi);   // (the rows are already sorted)
                if (i == 1 || i >= S - E + 2) ++cnt;
            }
            c.mortar_active[i - 1] = cnt;
        }
    }
    // viscous runs: at each stage the inactive face neighbours of the active
    // prefix (a ring), whose BR1 gradients enter the active elements' viscous
    // interface fluxes; sorted by element for locality
    c.ring.clear();
    c.ring_off.assign(S + 1, 0);
    if (c.viscous) {
        std::vector<int32_t> pos(NE);
        for (size_t j = 0; j < NE; ++j) pos[c.elist[j]] = (int32_t)j;
        std::vector<char> mark(NE, 0);
        for (int i = 0; i < S; ++i) {
            c.ring_off[i] = (int32_t)c.ring.size();
            std::vector<int32_t> r;
            for (int j = 0; j < c.n_active[i]; ++j) {
                const size_t e = (size_t)c.elist[j];
                for (int f = 0; f < NF; ++f) {
                    const int32_t nb = c.nbr[e * NF + f];
                    if (pos[nb] >= c.n_active[i] && !mark[nb]) {
                        mark[nb] = 1;
                        r.push_back(nb);
                    }
                }
            }
            std::sort(r.begin(), r.end());
            for (int32_t nb : r) mark[nb] = 0;
            c.ring.insert(c.ring.end(), r.begin(), r.end());
        }
        c.ring_off[S] = (int32_t)c.ring.size();
    }
    // fused direction: with b_i != 0 only at the first, penultimate and last
    // stage (all archetypes), d = b_1 K_1 + b_m K_{S-1} + b_S K_S is formed at
    // the last stage, where K_1 and K_{S-1} are read for the stage row anyway
    c.d_fused = c.opt.fuse_direction != 0;
    for (int k = 0; k < n; ++k) {
        const Instance &I = c.inst[k];
        for (int j = 1; j < I.S - 2; ++j)
            if (I.b[j] != 0.0) c.d_fused = false;
        if (I.S < 2) c.d_fused = false;
    }
    c.any_b.assign(S, 0);
    c.d_read.assign(S, 0);
    for (int k = 0; k < n; ++k) {
        const Instance &I = c.inst[k];
        bool seen_b = false;
        for (int j = 0; j < I.S; ++j)
            if (I.b[j] != 0.0) {
                c.any_b[j == 0 ? 0 : S - I.S + j] = 1;
                if (seen_b && !c.d_fused) c.d_read[j == 0 ? 0 : S - I.S + j] = 1;
                seen_b = true;
            }
    }
    make_chunks(c, 152);
    return PERRK_OK;
}

// Relaxation work chunks: contiguous element ranges inside one instance, sized
// so that a pass has at least ~4 blocks per SM (nodes per chunk between 128
// and 4096).
void make_chunks(Ctx &c, int sm_count) {
    const int NP = c.NP;
    const long long nodes = (long long)c.n_elem * NP;
    long long target = nodes / (4LL * std::max(1, sm_count));
    target = std::max(128LL, std::min(4096LL, target));
    c.chunk_elems = std::max(1, (int)(target / NP));
    c.chunk_inst.clear();
    c.chunk_e0.clear();
    c.chunk_e1.clear();
    for (int k = 0; k < c.n_inst; ++k) {
        Instance &I = c.inst[k];
        I.chunk0 = (int)c.chunk_inst.size();
        for (int e = 0; e < I.n_elem; e += c.chunk_elems) {
            c.chunk_inst.push_back(k);
            c.chunk_e0.push_back(I.elem0 + e);
            c.chunk_e1.push_back(I.elem0 + std::min(I.n_elem, e + c.chunk_elems));
        }
        I.n_chunks = (int)c.chunk_inst.size() - I.chunk0;
    }
}

void stage_coefficients(const Ctx &c, std::vector<StageCoef> &coef, std::vector<StageCoefF> &coef_f) {
    coef.assign((size_t)c.S * c.n_gp, StageCoef{0, 0, 0, 0, 0, 0, 0});
    coef_f.assign((size_t)c.S * c.n_gp, StageCoefF{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0});
    auto split = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (const Instance &I : c.inst) {
        int first_b = -1;
        for (int j = 0; j < I.S; ++j)
            if (I.b[j] != 0.0) {
                first_b = j;
                break;
            }
        for (int i = 0; i < c.S; ++i) {
            int j = (i == 0) ? 0 : i - (c.S - I.S);  // local 0-based stage
            if (j < 0) continue;                     // instance idle at this global stage
            if (i > 0 && j == 0) continue;
            for (int r = 0; r < I.R; ++r) {
                StageCoef &sc = coef[(size_t)i * c.n_gp + I.gp0 + r];
                sc.a1 = I.dt * I.a1[r * I.S + j];
                sc.asub = I.dt * I.asub[r * I.S + j];
                sc.b = I.b[j];
                sc.first_b = (j == first_b) ? 1.0 : 0.0;
                const bool last = c.d_fused && j == I.S - 1;
                sc.b1 = last ? I.b[0] : 0.0;
                sc.bm = (last && I.S - 2 > 0) ? I.b[I.S - 2] : 0.0;
                sc.d_final = last ? 1.0 : 0.0;
                StageCoefF &cf = coef_f[(size_t)i * c.n_gp + I.gp0 + r];
                cf.a1 = (float)sc.a1;
                cf.asub = (float)sc.asub;
                split(sc.b, cf.b_hi, cf.b_lo);
                cf.has_b = sc.b != 0.0 ? 1 : 0;
                cf.first_b = j == first_b ? 1 : 0;
                cf.d_final = last ? 1 : 0;
                split(sc.b1, cf.b1_hi, cf.b1_lo);
                split(sc.bm, cf.bm_hi, cf.bm_lo);
            }
        }
    }
}

// Tables of the double-float logarithm: for F_j = 1 + j/128 (j = 0..128)
// log F_j and 1/F_j in long double, each split into a float pair; constants
// log 2, (slots 2-3 unused), gamma - 1 and gamma as float pairs.
static void split2(long double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (long double)hi);
}

void df_tables(double gamma_gas, std::vector<float> &tab, std::vector<float> &consts) {
    tab.assign(129 * 4, 0.0f);
    for (int j = 0; j <= 128; ++j) {
        const long double F = 1.0L + j / 128.0L;
        split2(std::log(F), tab[4 * j + 0], tab[4 * j + 1]);
        split2(1.0L / F, tab[4 * j + 2], tab[4 * j + 3]);
    }
    consts.assign(8, 0.0f);
    split2(std::log(2.0L), consts[0], consts[1]);
    split2((long double)gamma_gas - 1.0L, consts[4], consts[5]);
    split2((long double)gamma_gas, consts[6], consts[7]);
}

}  // namespace perrk

extern "C" perrk_status perrk_build_tableau(int p, int R, const int32_t *E, int S_cap, int *S_out, double *c, double *b,
                                           double *a1, double *asub) {
    using namespace perrk;
    if (p < 2 || p > 4 || R < 1 || R > kMaxR || !E || !S_out || !c || !b || !a1 || !asub) {
        set_error("build_tableau: p must be 2..4, R 1.." + std::to_string(kMaxR) + ", pointers non-null");
        return PERRK_INVALID_ARG;
    }
    int S = 0;
    for (int r = 0; r < R; ++r) {
        if (E[r] < min_E(p)) {
            set_error("build_tableau: E[" + std::to_string(r) + "] = " + std::to_string(E[r]) +
                      " is below the archetype minimum " + std::to_string(min_E(p)));
            return PERRK_INVALID_ARG;
        }
        S = std::max(S, (int)E[r]);
    }
    if (S > S_cap || S > 64) {
        set_error("build_tableau: S = " + std::to_string(S) + " exceeds the output capacity or 64");
        return PERRK_INVALID_ARG;
    }
    *S_out = S;
    // shared abscissae and weights (1-based stage i -> index i-1)
    std::vector<double> cc(S + 1, 0.0);
    for (int i = 1; i <= S; ++i) {
        if (p == 2) cc[i] = (i - 1) / (2.0 * (S - 1));
        else if (p == 3) cc[i] = (i <= S - 2) ? (S > 3 ? (i - 1) / (double)(S - 3) : 0.0) : (i == S - 1 ? 1.0 : 0.5);
        else cc[i] = (i == 1) ? 0.0 : (i <= S - 3 ? 1.0 : 0.0);
    }
    if (p == 4) {
        cc[S - 2] = 0.479274057836310;
        cc[S - 1] = 0.5 + std::sqrt(3.0) / 6.0;
        cc[S] = 0.5 - std::sqrt(3.0) / 6.0;
    }
    for (int i = 1; i <= S; ++i) {
        c[i - 1] = cc[i];
        b[i - 1] = 0.0;
    }
    if (p == 2) b[S - 1] = 1.0;
    else if (p == 3) {
        b[0] = 1.0 / 6.0;
        b[S - 2] = 1.0 / 6.0;
        b[S - 1] = 2.0 / 3.0;
    } else {
        b[S - 2] = 0.5;
        b[S - 1] = 0.5;
    }
    for (int r = 0; r < R; ++r) {
        const int Er = E[r], first = S - Er + 2;
        std::vector<double> sub(S + 1, 0.0);  // a_{i,i-1} for rows first+1 .. S
        if (p == 2) {
            // stability polynomial coefficient of z^j is c_{S-j+2} prod_{m=S-j+3}^S a_m; match 1/j!
            double prod = 1.0, fact = 2.0;
            for (int j = 3; j <= Er; ++j) {
                fact *= j;
                const int m = S - j + 3;
                sub[m] = (1.0 / fact) / (cc[S - j + 2] * prod);
                prod *= sub[m];
            }
        } else if (p == 3) {
            for (int i = first + 1; i <= S - 2; ++i) sub[i] = cc[i] / 8.0;
            if (S - 1 > first) sub[S - 1] = 0.25;
            sub[S] = (1.0 - sub[S - 1]) / 4.0;  // order-3 condition b^T A c = 1/6
        } else {
            for (int i = first + 1; i <= S - 3; ++i) sub[i] = cc[i] / 8.0;
            sub[S - 2] = 0.114851811257441 / cc[S - 3];
            sub[S - 1] = 0.648906880894214;
            sub[S] = 0.0283121635129678;
        }
        for (int i = 1; i <= S; ++i) {
            double a = (i > first) ? sub[i] : 0.0;
            if (i == 1) a = 0.0;
            if (i == 2) a = 0.0;  // the only earlier stage is K_1: a row (c_2, 0)
            a1[r * S + i - 1] = cc[i] - a;
            asub[r * S + i - 1] = a;
        }
    }
    return PERRK_OK;
}
