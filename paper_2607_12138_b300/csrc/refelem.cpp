// Reference-element tables for the BRAS library (host side, computed once per setup).
//
// What is computed: the reference mass blocks R_ab[i][j] = int_Kref phi_i^a phi_j^b of the
// nodal basis of each element family, from which every physical element matrix follows by
// the Piola pullbacks of Sec. 2.4 (Eq. piola_mass_pullbacks):
//   H1:      M_K = |det J| R_00
//   H(curl): M_K = sum_ab G_ab R_ab,  G = |det J| J^{-1} J^{-T}
//   H(div):  M_K = sum_ab G_ab R_ab,  G = J^T J / |det J|
//
// How (this library's own construction):
//   * integrals by collapsed (Duffy) tensor Gauss-Legendre rules, exact for the degrees used;
//   * Lagrange: Silvester's product form of the nodal basis in barycentric coordinates,
//     phi_alpha = prod_i prod_{m < alpha_i} (p lambda_i - m) / (m + 1);
//   * Lagrange at GLL-based nodes (the spectral nodal variant of Sec. 3): the recursive nodes
//     of Isaac (2020) on the Gauss-Lobatto-Legendre points of [0, 1] (Newton iterations on
//     P_n'), the nodal basis by a long-double inverse of the monomial Vandermonde matrix;
//   * Nedelec / Raviart-Thomas: the Arnold-Falk-Winther geometric bases of P_k^- Lambda^1
//     and P_k^- Lambda^2 (lambda^alpha times Whitney forms, alpha_m = 0 below the first
//     vertex of the form) as a spanning basis, dualised against the documented dof
//     functionals (edge Legendre moments, face moments against mean-orthonormal
//     polynomials, interior moments) by an LU solve in long double;
//   * second kind (N2curl_k / BDM_k): the monomial vectors of P_k^d dualised the same way, with
//     edge moments up to L_k, BDM face moments against P_k and the remaining face / interior
//     moments taken against the nodal bases of the lower-order first-kind elements above.
#include "refelem.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <vector>

namespace bras {
namespace {

struct QP { double x[3]; double w; };

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        long double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        long double dp = 1;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (std::fabs((double)dz) < 1e-19) break;
        }
        x[i] = (double)((1 - z) / 2);
        w[i] = (double)(1 / ((1 - z * z) * dp * dp));   // 2/((1-z^2)p'^2) scaled by 1/2
    }
}

constexpr int kQuad = 9;   // 9-point rules: exact to degree 17 per collapsed direction

std::vector<QP> segment_rule() {
    std::vector<double> x, w;
    gauss_legendre01(kQuad, x, w);
    std::vector<QP> q;
    for (int i = 0; i < kQuad; ++i) q.push_back({{x[i], 0, 0}, w[i]});
    return q;
}

std::vector<QP> triangle_rule() {   // (s, t) = (u, v (1-u)), weight (1-u)
    std::vector<double> x, w;
    gauss_legendre01(kQuad, x, w);
    std::vector<QP> q;
    for (int i = 0; i < kQuad; ++i)
        for (int j = 0; j < kQuad; ++j)
            q.push_back({{x[i], x[j] * (1 - x[i]), 0}, w[i] * w[j] * (1 - x[i])});
    return q;
}

std::vector<QP> tet_rule() {        // (x, y, z) = (u, v (1-u), w (1-u)(1-v))
    std::vector<double> x, w;
    gauss_legendre01(kQuad, x, w);
    std::vector<QP> q;
    for (int i = 0; i < kQuad; ++i)
        for (int j = 0; j < kQuad; ++j)
            for (int k = 0; k < kQuad; ++k) {
                double u = x[i], v = x[j], s = x[k];
                q.push_back({{u, v * (1 - u), s * (1 - u) * (1 - v)},
                             w[i] * w[j] * w[k] * (1 - u) * (1 - u) * (1 - v)});
            }
    return q;
}

// barycentric coordinates on the reference simplex, vertices 0, e_1, .., e_d
void bary(int dim, const double* x, double* lam) {
    double s = 0;
    for (int i = 0; i < dim; ++i) { lam[i + 1] = x[i]; s += x[i]; }
    lam[0] = 1 - s;
}

void bary_grad(int i, double g[3]) {
    for (int c = 0; c < 3; ++c) g[c] = (i == 0) ? -1.0 : (c == i - 1 ? 1.0 : 0.0);
}

// multi-indices of length m and sum s, ascending lexicographic
void compositions(int m, int s, std::vector<std::vector<int>>& out) {
    std::vector<int> a(m, 0);
    out.clear();
    std::function<void(int, int)> rec = [&](int pos, int left) {
        if (pos == m - 1) { a[pos] = left; out.push_back(a); return; }
        for (int v = 0; v <= left; ++v) { a[pos] = v; rec(pos + 1, left - v); }
    };
    rec(0, s);
}

// ---- Lagrange -------------------------------------------------------------------------
double silvester(int p, const std::vector<int>& alpha, const double* lam) {
    double v = 1;
    for (size_t i = 0; i < alpha.size(); ++i)
        for (int m = 0; m < alpha[i]; ++m) v *= (p * lam[i] - m) / (m + 1);
    return v;
}

int build_lagrange(int dim, int p, RefTables* out) {
    std::vector<std::vector<int>> nodes;
    compositions(dim + 1, p, nodes);             // ascending lexicographic in (a_0..a_d)
    const int n = (int)nodes.size();
    auto rule = dim == 3 ? tet_rule() : triangle_rule();
    out->nloc = n;
    out->ncomp = 1;
    out->R.assign((size_t)n * n, 0.0);
    std::vector<double> phi(n);
    for (const QP& q : rule) {
        double lam[4];
        bary(dim, q.x, lam);
        for (int i = 0; i < n; ++i) phi[i] = silvester(p, nodes[i], lam);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) out->R[(size_t)i * n + j] += q.w * phi[i] * phi[j];
    }
    return 0;
}

// ---- Lagrange at GLL-based nodes --------------------------------------------------------
// n + 1 Gauss-Lobatto-Legendre points of [0, 1], ascending: the end points and the roots of
// P_n', found by Newton's method from the Chebyshev-Gauss-Lobatto points, with P_n and P_n'
// from the three-term recurrence and P_n'' from Legendre's equation.
std::vector<long double> gll_points01(int n) {
    std::vector<long double> x(n + 1);
    x[0] = 0;
    x[n] = 1;
    for (int j = 1; j < n; ++j) {
        long double t = -std::cos(M_PI * (long double)j / n);
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = t;   // P_{k-1}, P_k
            for (int k = 1; k < n; ++k) {
                const long double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            const long double dp = n * (t * p1 - p0) / (t * t - 1);              // P_n'
            const long double d2p = (2 * t * dp - n * (n + 1) * p1) / (1 - t * t);  // P_n''
            const long double step = dp / d2p;
            t -= step;
            if (std::fabs(step) < 1e-19L) break;
        }
        x[j] = (t + 1) / 2;
    }
    return x;
}

// Barycentric coordinates of the recursive node of multi-index a: the weighted mean of the
// facet nodes b(a without a_i) embedded with a zero at position i, weights x_{n, n - a_i}
// (n = |a|); one coordinate 1 for a single index.
std::vector<long double> recursive_node(const std::vector<int>& a) {
    const int d = (int)a.size() - 1;
    int n = 0;
    for (int v : a) n += v;
    if (d == 0) return {1.0L};
    if (n == 0) return std::vector<long double>(d + 1, 1.0L / (d + 1));   // weight 0 below
    const std::vector<long double> x = gll_points01(n);
    std::vector<long double> acc(d + 1, 0.0L);
    long double wsum = 0;
    for (int i = 0; i <= d; ++i) {
        std::vector<int> sub;
        for (int j = 0; j <= d; ++j)
            if (j != i) sub.push_back(a[j]);
        const std::vector<long double> bs = recursive_node(sub);
        const long double w = x[n - a[i]];
        for (int j = 0, k = 0; j <= d; ++j) acc[j] += w * (j == i ? 0.0L : bs[k++]);
        wsum += w;
    }
    for (auto& v : acc) v /= wsum;
    return acc;
}

bool lu_inverse(std::vector<long double> A, int n, std::vector<long double>& inv);

int build_lagrange_gll(int dim, int p, RefTables* out) {
    std::vector<std::vector<int>> nodes;
    compositions(dim + 1, p, nodes);             // ascending lexicographic, as the equispaced nodes
    const int n = (int)nodes.size();
    // monomials x^a y^b z^c of total degree <= p
    std::vector<std::array<int, 3>> mono;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b + a <= p; ++b)
            for (int c = 0; c + a + b <= p; ++c)
                if (dim == 3 || c == 0) mono.push_back({a, b, c});
    if ((int)mono.size() != n) return -1;
    auto eval_mono = [&](const long double* x, std::vector<long double>& m) {
        m.resize(n);
        for (int j = 0; j < n; ++j) {
            long double v = 1;
            for (int c = 0; c < dim; ++c)
                for (int e = 0; e < mono[j][c]; ++e) v *= x[c];
            m[j] = v;
        }
    };
    // Vandermonde V[i][j] = m_j(node_i); the nodal basis phi_i = sum_j m_j C[j][i], C = V^{-1}
    std::vector<long double> V((size_t)n * n), C, m;
    for (int i = 0; i < n; ++i) {
        const std::vector<long double> lam = recursive_node(nodes[i]);
        long double x[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) x[c] = lam[c + 1];   // vertices 0, e_1, .., e_d
        eval_mono(x, m);
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = m[j];
    }
    if (!lu_inverse(V, n, C)) return -1;
    auto rule = dim == 3 ? tet_rule() : triangle_rule();
    out->nloc = n;
    out->ncomp = 1;
    out->R.assign((size_t)n * n, 0.0);
    std::vector<long double> phi(n);
    std::vector<long double> acc((size_t)n * n, 0.0L);
    for (const QP& q : rule) {
        const long double x[3] = {q.x[0], q.x[1], q.x[2]};
        eval_mono(x, m);
        for (int i = 0; i < n; ++i) {
            long double v = 0;
            for (int j = 0; j < n; ++j) v += m[j] * C[(size_t)j * n + i];
            phi[i] = v;
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) acc[(size_t)i * n + j] += (long double)q.w * phi[i] * phi[j];
    }
    for (size_t i = 0; i < acc.size(); ++i) out->R[i] = (double)acc[i];
    return 0;
}

// ---- vector elements ------------------------------------------------------------------
using Vec3 = std::array<double, 3>;
// Values of every nodal basis function of an element at a reference point (3 components; the
// third is zero on triangles).
using BasisEval = std::function<void(const double* x, std::vector<Vec3>& vals)>;

struct SpanFn {            // lambda^alpha * form(vertices)
    std::array<int, 4> alpha;
    std::array<int, 3> v;  // edge (v0, v1) or face (v0, v1, v2)
};

Vec3 cross(const Vec3& a, const Vec3& b) {
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}

Vec3 eval_span(bool curl, const SpanFn& f, const double* x) {
    double lam[4];
    bary(3, x, lam);
    double pw = 1;
    for (int i = 0; i < 4; ++i)
        for (int m = 0; m < f.alpha[i]; ++m) pw *= lam[i];
    Vec3 g[4];
    for (int i = 0; i < 4; ++i) { double t[3]; bary_grad(i, t); g[i] = {t[0], t[1], t[2]}; }
    Vec3 r{0, 0, 0};
    if (curl) {            // Whitney edge form lam_a grad lam_b - lam_b grad lam_a
        int a = f.v[0], b = f.v[1];
        for (int c = 0; c < 3; ++c) r[c] = lam[a] * g[b][c] - lam[b] * g[a][c];
    } else {               // Whitney face form lam_a gb x gc - lam_b ga x gc + lam_c ga x gb
        int a = f.v[0], b = f.v[1], c = f.v[2];
        Vec3 bc = cross(g[b], g[c]), ac = cross(g[a], g[c]), ab = cross(g[a], g[b]);
        for (int d = 0; d < 3; ++d) r[d] = lam[a] * bc[d] - lam[b] * ac[d] + lam[c] * ab[d];
    }
    for (int c = 0; c < 3; ++c) r[c] *= pw;
    return r;
}

std::vector<SpanFn> afw_span(bool curl, int k) {
    std::vector<SpanFn> out;
    std::vector<std::vector<int>> al;
    compositions(4, k - 1, al);
    if (curl) {
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                for (auto& m : al) {
                    bool ok = true;
                    for (int i = 0; i < a; ++i) ok &= (m[i] == 0);
                    if (ok) out.push_back({{m[0], m[1], m[2], m[3]}, {a, b, -1}});
                }
    } else {
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                for (int c = b + 1; c < 4; ++c)
                    for (auto& m : al) {
                        bool ok = true;
                        for (int i = 0; i < a; ++i) ok &= (m[i] == 0);
                        if (ok) out.push_back({{m[0], m[1], m[2], m[3]}, {a, b, c}});
                    }
    }
    return out;
}

// Gram-Schmidt (mean inner product) of monomials sampled at quadrature points.
// Returns values [n_poly][n_pts].
std::vector<std::vector<double>> orthonormal_values(const std::vector<QP>& rule, double measure,
                                                    const std::vector<std::array<int, 3>>& monos) {
    std::vector<std::vector<double>> q;
    for (const auto& e : monos) {
        std::vector<double> v(rule.size());
        for (size_t i = 0; i < rule.size(); ++i)
            v[i] = std::pow(rule[i].x[0], e[0]) * std::pow(rule[i].x[1], e[1]) * std::pow(rule[i].x[2], e[2]);
        for (const auto& prev : q) {          // classical GS against the finished ones
            double dot = 0;
            for (size_t i = 0; i < rule.size(); ++i) dot += rule[i].w * v[i] * prev[i];
            dot /= measure;
            for (size_t i = 0; i < rule.size(); ++i) v[i] -= dot * prev[i];
        }
        double nn = 0;
        for (size_t i = 0; i < rule.size(); ++i) nn += rule[i].w * v[i] * v[i];
        nn = std::sqrt(nn / measure);
        for (double& t : v) t /= nn;
        q.push_back(v);
    }
    return q;
}

// triangle test monomials s^i t^j: degree ascending, then power of t ascending
std::vector<std::array<int, 3>> triangle_monos(int deg) {
    std::vector<std::array<int, 3>> m;
    for (int d = 0; d <= deg; ++d)
        for (int j = 0; j <= d; ++j) m.push_back({d - j, j, 0});
    return m;
}

// tetrahedron monomials: degree ascending, then descending lexicographic exponent tuple
std::vector<std::array<int, 3>> tet_monos(int deg) {
    std::vector<std::array<int, 3>> m;
    for (int d = 0; d <= deg; ++d) {
        std::vector<std::array<int, 3>> lvl;
        for (int a = 0; a <= d; ++a)
            for (int b = 0; a + b <= d; ++b) lvl.push_back({a, b, d - a - b});
        std::sort(lvl.begin(), lvl.end(), [](auto& u, auto& v) { return u > v; });
        m.insert(m.end(), lvl.begin(), lvl.end());
    }
    return m;
}

double shifted_legendre(int j, double u) {
    double z = 2 * u - 1, p0 = 1, p1 = z;
    if (j == 0) return 1;
    for (int k = 2; k <= j; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

bool lu_inverse(std::vector<long double> A, int n, std::vector<long double>& inv) {
    std::vector<int> piv(n);
    for (int i = 0; i < n; ++i) piv[i] = i;
    for (int k = 0; k < n; ++k) {
        int m = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs((double)A[(size_t)i * n + k]) > std::fabs((double)A[(size_t)m * n + k])) m = i;
        if (A[(size_t)m * n + k] == 0) return false;
        if (m != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)m * n + j]);
            std::swap(piv[k], piv[m]);
        }
        for (int i = k + 1; i < n; ++i) {
            long double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        }
    }
    inv.assign((size_t)n * n, 0);
    for (int c = 0; c < n; ++c) {
        std::vector<long double> y(n);
        for (int i = 0; i < n; ++i) {
            long double s = (piv[i] == c) ? 1 : 0;
            for (int j = 0; j < i; ++j) s -= A[(size_t)i * n + j] * y[j];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            long double s = y[i];
            for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * y[j];
            y[i] = s / A[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = y[i];
    }
    return true;
}

const int kEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kFaces[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
const double kVert[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

int build_vector(bool curl, int k, RefTables* out, BasisEval* ev = nullptr) {
    const auto span = afw_span(curl, k);
    const int n = (int)span.size();
    const int expect = curl ? k * (k + 2) * (k + 3) / 2 : k * (k + 1) * (k + 3) / 2;
    if (n != expect) return -1;
    const auto seg = segment_rule();
    const auto tri = triangle_rule();
    const auto tet = tet_rule();
    // functional rows A[i][j] = l_i(span_j)
    std::vector<long double> A;
    A.reserve((size_t)n * n);
    auto push_row = [&](auto&& fn) {   // fn(span index) -> value
        for (int j = 0; j < n; ++j) A.push_back((long double)fn(j));
    };
    if (curl) {
        for (auto& e : kEdges) {
            Vec3 tau;
            for (int c = 0; c < 3; ++c) tau[c] = kVert[e[1]][c] - kVert[e[0]][c];
            for (int jm = 0; jm < k; ++jm)
                push_row([&](int j) {
                    double s = 0;
                    for (const QP& q : seg) {
                        double x[3];
                        for (int c = 0; c < 3; ++c) x[c] = kVert[e[0]][c] + q.x[0] * tau[c];
                        Vec3 v = eval_span(true, span[j], x);
                        s += q.w * (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2]) * shifted_legendre(jm, q.x[0]);
                    }
                    return s;
                });
        }
    }
    const int fdeg = curl ? k - 2 : k - 1;
    if (fdeg >= 0) {
        auto fq = orthonormal_values(tri, 0.5, triangle_monos(fdeg));
        for (auto& f : kFaces) {
            Vec3 t1, t2;
            for (int c = 0; c < 3; ++c) {
                t1[c] = kVert[f[1]][c] - kVert[f[0]][c];
                t2[c] = kVert[f[2]][c] - kVert[f[0]][c];
            }
            std::vector<Vec3> dirs = curl ? std::vector<Vec3>{t1, t2} : std::vector<Vec3>{cross(t1, t2)};
            for (size_t r = 0; r < fq.size(); ++r)
                for (const Vec3& d : dirs)
                    push_row([&](int j) {
                        double s = 0;
                        for (size_t qi = 0; qi < tri.size(); ++qi) {
                            double x[3];
                            for (int c = 0; c < 3; ++c)
                                x[c] = kVert[f[0]][c] + tri[qi].x[0] * t1[c] + tri[qi].x[1] * t2[c];
                            Vec3 v = eval_span(curl, span[j], x);
                            s += tri[qi].w * (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) * fq[r][qi];
                        }
                        return s;
                    });
        }
    }
    const int ideg = curl ? k - 3 : k - 2;
    if (ideg >= 0) {
        auto iq = orthonormal_values(tet, 1.0 / 6.0, tet_monos(ideg));
        for (size_t r = 0; r < iq.size(); ++r)
            for (int comp = 0; comp < 3; ++comp)
                push_row([&](int j) {
                    double s = 0;
                    for (size_t qi = 0; qi < tet.size(); ++qi)
                        s += tet[qi].w * eval_span(curl, span[j], tet[qi].x)[comp] * iq[r][qi];
                    return s;
                });
    }
    if ((int)A.size() != n * n) return -2;
    std::vector<long double> C;
    if (!lu_inverse(A, n, C)) return -3;
    if (ev)
        *ev = [span, C, n, curl](const double* x, std::vector<Vec3>& vals) {
            std::vector<Vec3> sv(n);
            for (int j = 0; j < n; ++j) sv[j] = eval_span(curl, span[j], x);
            vals.assign(n, Vec3{0, 0, 0});
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    long double acc = 0;
                    for (int j = 0; j < n; ++j) acc += (long double)sv[j][c] * C[(size_t)j * n + i];
                    vals[i][c] = (double)acc;
                }
        };
    // nodal basis phi_i = sum_j span_j C[j][i]; R_ab = int phi^a phi^b
    out->nloc = n;
    out->ncomp = 3;
    out->R.assign((size_t)9 * n * n, 0.0);
    std::vector<double> sv((size_t)n * 3), ph((size_t)n * 3);
    for (const QP& q : tet) {
        for (int j = 0; j < n; ++j) {
            Vec3 v = eval_span(curl, span[j], q.x);
            for (int c = 0; c < 3; ++c) sv[(size_t)j * 3 + c] = v[c];
        }
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) {
                long double s = 0;
                for (int j = 0; j < n; ++j) s += (long double)sv[(size_t)j * 3 + c] * C[(size_t)j * n + i];
                ph[(size_t)i * 3 + c] = (double)s;
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double* R = &out->R[(size_t)(a * 3 + b) * n * n];
                for (int i = 0; i < n; ++i) {
                    double wa = q.w * ph[(size_t)i * 3 + a];
                    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] += wa * ph[(size_t)j * 3 + b];
                }
            }
    }
    if (!curl) {
        // divergence block of the mixed Poisson pair RT_k / DG_{k-1}: the span's divergence in
        // closed form, div(lambda^alpha W_abc) = grad(lambda^alpha) . W_abc + 3 lambda^alpha
        // grad lambda_a . (grad lambda_b x grad lambda_c), against the mean-orthonormal
        // polynomials of degree <= k - 1, by the tetrahedral rule
        const auto chi = orthonormal_values(tet, 1.0 / 6.0, tet_monos(k - 1));
        const int nq = (int)chi.size();
        out->nq = nq;
        out->Bdiv.assign((size_t)nq * n, 0.0);
        Vec3 g[4];
        for (int i = 0; i < 4; ++i) {
            double t[3];
            bary_grad(i, t);
            g[i] = {t[0], t[1], t[2]};
        }
        std::vector<double> dv(n);
        for (size_t qi = 0; qi < tet.size(); ++qi) {
            double lam[4];
            bary(3, tet[qi].x, lam);
            for (int j = 0; j < n; ++j) {
                const SpanFn& f = span[j];
                const int a = f.v[0], b = f.v[1], c = f.v[2];
                double pw = 1;
                for (int m = 0; m < 4; ++m)
                    for (int e = 0; e < f.alpha[m]; ++e) pw *= lam[m];
                Vec3 grad_pw{0, 0, 0};
                for (int m = 0; m < 4; ++m) {
                    if (f.alpha[m] == 0) continue;
                    double t = f.alpha[m];
                    for (int mm = 0; mm < 4; ++mm)
                        for (int e = 0; e < f.alpha[mm] - (mm == m ? 1 : 0); ++e) t *= lam[mm];
                    for (int d = 0; d < 3; ++d) grad_pw[d] += t * g[m][d];
                }
                Vec3 W{0, 0, 0};
                const Vec3 bc = cross(g[b], g[c]), ac = cross(g[a], g[c]), ab = cross(g[a], g[b]);
                for (int d = 0; d < 3; ++d) W[d] = lam[a] * bc[d] - lam[b] * ac[d] + lam[c] * ab[d];
                const double divW = 3.0 * (g[a][0] * bc[0] + g[a][1] * bc[1] + g[a][2] * bc[2]);
                dv[j] = grad_pw[0] * W[0] + grad_pw[1] * W[1] + grad_pw[2] * W[2] + pw * divW;
            }
            for (int jj = 0; jj < n; ++jj) {   // divergence of the nodal function jj
                long double d = 0;
                for (int j = 0; j < n; ++j) d += (long double)dv[j] * C[(size_t)j * n + jj];
                for (int i = 0; i < nq; ++i) out->Bdiv[(size_t)i * n + jj] += tet[qi].w * (double)d * chi[i][qi];
            }
        }
    }
    return 0;
}

// ---- vector elements on triangles ----------------------------------------------------------
// N1curl_k: the geometric basis lambda^alpha (lambda_a grad lambda_b - lambda_b grad lambda_a),
// alpha of size k - 1 with alpha_m = 0 below the first vertex a of the edge; RT_k: the same
// functions rotated by R v = (v_y, -v_x).  Dofs: edge moments of v . t (N1curl) or v . R t (RT)
// against L_j, j < k, t = v_b - v_a; interior moments of the two components against the
// mean-orthonormal polynomials of degree <= k - 2 (q outer, component inner).  Tables are in the
// three-component layout of the tetrahedral families with a zero third component.
struct Span2 {
    std::array<int, 3> alpha;
    int a, b;
};

Vec3 eval_span2(bool curl, const Span2& f, const double* x) {
    double lam[3];
    bary(2, x, lam);
    double pw = 1;
    for (int i = 0; i < 3; ++i)
        for (int m = 0; m < f.alpha[i]; ++m) pw *= lam[i];
    const double g[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
    const double w0 = lam[f.a] * g[f.b][0] - lam[f.b] * g[f.a][0];
    const double w1 = lam[f.a] * g[f.b][1] - lam[f.b] * g[f.a][1];
    if (curl) return {w0 * pw, w1 * pw, 0.0};
    return {w1 * pw, -w0 * pw, 0.0};
}

int build_vector_2d(bool curl, int k, RefTables* out, BasisEval* ev = nullptr) {
    const int kE[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    const double kV[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    std::vector<Span2> span;
    std::vector<std::vector<int>> al;
    compositions(3, k - 1, al);
    for (auto& e : kE)
        for (auto& m : al) {
            bool ok = true;
            for (int i = 0; i < e[0]; ++i) ok &= (m[i] == 0);
            if (ok) span.push_back({{m[0], m[1], m[2]}, e[0], e[1]});
        }
    const int n = (int)span.size();
    if (n != k * (k + 2)) return -1;
    const auto seg = segment_rule();
    const auto tri = triangle_rule();
    std::vector<long double> A;
    A.reserve((size_t)n * n);
    for (auto& e : kE) {
        const double t[2] = {kV[e[1]][0] - kV[e[0]][0], kV[e[1]][1] - kV[e[0]][1]};
        const double d[2] = {curl ? t[0] : t[1], curl ? t[1] : -t[0]};
        for (int jm = 0; jm < k; ++jm)
            for (int j = 0; j < n; ++j) {
                double acc = 0;
                for (const QP& q : seg) {
                    const double x[3] = {kV[e[0]][0] + q.x[0] * t[0], kV[e[0]][1] + q.x[0] * t[1], 0};
                    const Vec3 v = eval_span2(curl, span[j], x);
                    acc += q.w * (v[0] * d[0] + v[1] * d[1]) * shifted_legendre(jm, q.x[0]);
                }
                A.push_back(acc);
            }
    }
    if (k >= 2) {
        auto iq = orthonormal_values(tri, 0.5, triangle_monos(k - 2));
        for (size_t r = 0; r < iq.size(); ++r)
            for (int comp = 0; comp < 2; ++comp)
                for (int j = 0; j < n; ++j) {
                    double acc = 0;
                    for (size_t qi = 0; qi < tri.size(); ++qi)
                        acc += tri[qi].w * eval_span2(curl, span[j], tri[qi].x)[comp] * iq[r][qi];
                    A.push_back(acc);
                }
    }
    if ((int)A.size() != n * n) return -2;
    std::vector<long double> C;
    if (!lu_inverse(A, n, C)) return -3;
    if (ev)
        *ev = [span, C, n, curl](const double* x, std::vector<Vec3>& vals) {
            std::vector<Vec3> sv(n);
            for (int j = 0; j < n; ++j) sv[j] = eval_span2(curl, span[j], x);
            vals.assign(n, Vec3{0, 0, 0});
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 2; ++c) {
                    long double acc = 0;
                    for (int j = 0; j < n; ++j) acc += (long double)sv[j][c] * C[(size_t)j * n + i];
                    vals[i][c] = (double)acc;
                }
        };
    out->nloc = n;
    out->ncomp = 3;
    out->R.assign((size_t)9 * n * n, 0.0);
    std::vector<double> sv((size_t)n * 2), ph((size_t)n * 2);
    for (const QP& q : tri) {
        for (int j = 0; j < n; ++j) {
            const Vec3 v = eval_span2(curl, span[j], q.x);
            sv[(size_t)j * 2] = v[0];
            sv[(size_t)j * 2 + 1] = v[1];
        }
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 2; ++c) {
                long double acc = 0;
                for (int j = 0; j < n; ++j) acc += (long double)sv[(size_t)j * 2 + c] * C[(size_t)j * n + i];
                ph[(size_t)i * 2 + c] = (double)acc;
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double* R = &out->R[(size_t)(a * 3 + b) * n * n];
                for (int i = 0; i < n; ++i) {
                    const double wa = q.w * ph[(size_t)i * 2 + a];
                    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] += wa * ph[(size_t)j * 2 + b];
                }
            }
    }
    return 0;
}

// ---- second-kind vector elements: N2curl_k (curl) and BDM_k (div), the full P_k^d -----------
// Spanning basis: the monomial vectors x^m e_c (c outer, monomials inner), dualised against
//   * edge moments of v . t (N2curl) or, on triangles, of v . (t_y, -t_x) (BDM) against L_j,
//     j = 0..k (one more than the first kind);
//   * BDM faces: moments of v . (t1 x t2) against the mean-orthonormal P_k of the face;
//   * N2curl faces (k >= 2): int_T v(x(s, t)) . (psi^s t1 + psi^t t2) ds dt over the nodal basis
//     psi of RT_{k-1} on the reference triangle, face outer;
//   * interior: int v . psi over the nodal basis psi of RT_{k-1} (N2curl, triangles), RT_{k-2}
//     (N2curl, tetrahedra, k >= 3) or N1curl_{k-1} (BDM, k >= 2), those bases built above.
int build_second_kind(int dim, bool curl, int k, RefTables* out) {
    const auto monos = dim == 3 ? tet_monos(k) : triangle_monos(k);
    const int nm = (int)monos.size(), n = dim * nm;
    auto span_val = [&](int j, const double* x) {   // x^m e_c
        const auto& m = monos[j % nm];
        double v = 1;
        for (int c = 0; c < dim; ++c)
            for (int e = 0; e < m[c]; ++e) v *= x[c];
        Vec3 r{0, 0, 0};
        r[j / nm] = v;
        return r;
    };
    const auto seg = segment_rule();
    const auto tri = triangle_rule();
    const auto tet = tet_rule();
    std::vector<long double> A;
    A.reserve((size_t)n * n);
    auto push_row = [&](auto&& fn) {
        for (int j = 0; j < n; ++j) A.push_back((long double)fn(j));
    };
    // interior moments against the nodal basis given by ev (reference cell quadrature)
    auto push_interior = [&](const BasisEval& ev, int npsi) {
        const auto& rule = dim == 3 ? tet : tri;
        std::vector<std::vector<Vec3>> pv(rule.size());
        for (size_t qi = 0; qi < rule.size(); ++qi) ev(rule[qi].x, pv[qi]);
        for (int r = 0; r < npsi; ++r)
            push_row([&](int j) {
                double s = 0;
                for (size_t qi = 0; qi < rule.size(); ++qi) {
                    const Vec3 v = span_val(j, rule[qi].x);
                    s += rule[qi].w * (v[0] * pv[qi][r][0] + v[1] * pv[qi][r][1] + v[2] * pv[qi][r][2]);
                }
                return s;
            });
    };
    if (dim == 2) {
        const int kE[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        const double kV[3][2] = {{0, 0}, {1, 0}, {0, 1}};
        for (auto& e : kE) {
            const double t[2] = {kV[e[1]][0] - kV[e[0]][0], kV[e[1]][1] - kV[e[0]][1]};
            const double d[2] = {curl ? t[0] : t[1], curl ? t[1] : -t[0]};
            for (int jm = 0; jm <= k; ++jm)
                push_row([&](int j) {
                    double acc = 0;
                    for (const QP& q : seg) {
                        const double x[3] = {kV[e[0]][0] + q.x[0] * t[0], kV[e[0]][1] + q.x[0] * t[1], 0};
                        const Vec3 v = span_val(j, x);
                        acc += q.w * (v[0] * d[0] + v[1] * d[1]) * shifted_legendre(jm, q.x[0]);
                    }
                    return acc;
                });
        }
        if (k >= 2) {
            RefTables tmp;
            BasisEval ev;
            if (build_vector_2d(!curl, k - 1, &tmp, &ev) != 0) return -4;   // RT_{k-1} / N1curl_{k-1}
            push_interior(ev, tmp.nloc);
        }
    } else {
        if (curl) {
            for (auto& e : kEdges) {
                Vec3 tau;
                for (int c = 0; c < 3; ++c) tau[c] = kVert[e[1]][c] - kVert[e[0]][c];
                for (int jm = 0; jm <= k; ++jm)
                    push_row([&](int j) {
                        double s = 0;
                        for (const QP& q : seg) {
                            double x[3];
                            for (int c = 0; c < 3; ++c) x[c] = kVert[e[0]][c] + q.x[0] * tau[c];
                            const Vec3 v = span_val(j, x);
                            s += q.w * (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2]) * shifted_legendre(jm, q.x[0]);
                        }
                        return s;
                    });
            }
            if (k >= 2) {
                RefTables tmp;
                BasisEval ev;
                if (build_vector_2d(false, k - 1, &tmp, &ev) != 0) return -4;   // RT_{k-1}, triangle
                std::vector<std::vector<Vec3>> pv(tri.size());
                for (size_t qi = 0; qi < tri.size(); ++qi) ev(tri[qi].x, pv[qi]);
                for (auto& f : kFaces) {
                    Vec3 t1, t2;
                    for (int c = 0; c < 3; ++c) {
                        t1[c] = kVert[f[1]][c] - kVert[f[0]][c];
                        t2[c] = kVert[f[2]][c] - kVert[f[0]][c];
                    }
                    for (int r = 0; r < tmp.nloc; ++r)
                        push_row([&](int j) {
                            double s = 0;
                            for (size_t qi = 0; qi < tri.size(); ++qi) {
                                double x[3];
                                for (int c = 0; c < 3; ++c)
                                    x[c] = kVert[f[0]][c] + tri[qi].x[0] * t1[c] + tri[qi].x[1] * t2[c];
                                const Vec3 v = span_val(j, x);
                                double w = 0;
                                for (int c = 0; c < 3; ++c) w += v[c] * (pv[qi][r][0] * t1[c] + pv[qi][r][1] * t2[c]);
                                s += tri[qi].w * w;
                            }
                            return s;
                        });
                }
            }
            if (k >= 3) {
                RefTables tmp;
                BasisEval ev;
                if (build_vector(false, k - 2, &tmp, &ev) != 0) return -4;   // RT_{k-2}
                push_interior(ev, tmp.nloc);
            }
        } else {
            auto fq = orthonormal_values(tri, 0.5, triangle_monos(k));
            for (auto& f : kFaces) {
                Vec3 t1, t2;
                for (int c = 0; c < 3; ++c) {
                    t1[c] = kVert[f[1]][c] - kVert[f[0]][c];
                    t2[c] = kVert[f[2]][c] - kVert[f[0]][c];
                }
                const Vec3 nrm = cross(t1, t2);
                for (size_t r = 0; r < fq.size(); ++r)
                    push_row([&](int j) {
                        double s = 0;
                        for (size_t qi = 0; qi < tri.size(); ++qi) {
                            double x[3];
                            for (int c = 0; c < 3; ++c)
                                x[c] = kVert[f[0]][c] + tri[qi].x[0] * t1[c] + tri[qi].x[1] * t2[c];
                            const Vec3 v = span_val(j, x);
                            s += tri[qi].w * (v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2]) * fq[r][qi];
                        }
                        return s;
                    });
            }
            if (k >= 2) {
                RefTables tmp;
                BasisEval ev;
                if (build_vector(true, k - 1, &tmp, &ev) != 0) return -4;   // N1curl_{k-1}
                push_interior(ev, tmp.nloc);
            }
        }
    }
    if ((int)A.size() != n * n) return -2;
    std::vector<long double> C;
    if (!lu_inverse(A, n, C)) return -3;
    out->nloc = n;
    out->ncomp = 3;
    out->R.assign((size_t)9 * n * n, 0.0);
    if (!curl && dim == 3) {
        // divergence block of the mixed Poisson pair BDM_k / DG_{k-1}: div(x^m e_c) =
        // m_c x^(m - e_c), against the mean-orthonormal polynomials of degree <= k - 1
        const auto chi = orthonormal_values(tet, 1.0 / 6.0, tet_monos(k - 1));
        const int nq = (int)chi.size();
        out->nq = nq;
        out->Bdiv.assign((size_t)nq * n, 0.0);
        std::vector<double> dv(n);
        for (size_t qi = 0; qi < tet.size(); ++qi) {
            const double* x = tet[qi].x;
            for (int j = 0; j < n; ++j) {
                const int c = j / nm;
                const auto& m = monos[j % nm];
                double v = 0;
                if (m[c] > 0) {
                    v = m[c];
                    for (int d = 0; d < 3; ++d)
                        for (int e = 0; e < m[d] - (d == c ? 1 : 0); ++e) v *= x[d];
                }
                dv[j] = v;
            }
            for (int jj = 0; jj < n; ++jj) {   // divergence of the nodal function jj
                long double d = 0;
                for (int j = 0; j < n; ++j) d += (long double)dv[j] * C[(size_t)j * n + jj];
                for (int i = 0; i < nq; ++i) out->Bdiv[(size_t)i * n + jj] += tet[qi].w * (double)d * chi[i][qi];
            }
        }
    }
    const auto& rule = dim == 3 ? tet : tri;
    std::vector<Vec3> sv(n), ph(n);
    for (const QP& q : rule) {
        for (int j = 0; j < n; ++j) sv[j] = span_val(j, q.x);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) {
                long double acc = 0;
                for (int j = 0; j < n; ++j) acc += (long double)sv[j][c] * C[(size_t)j * n + i];
                ph[i][c] = (double)acc;
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double* R = &out->R[(size_t)(a * 3 + b) * n * n];
                for (int i = 0; i < n; ++i) {
                    const double wa = q.w * ph[i][a];
                    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] += wa * ph[j][b];
                }
            }
    }
    return 0;
}

}  // namespace

int n_local(int dim, int space, int order, int basis) {
    if (basis < 0 || basis > 2 || (space != 0 && basis == 2)) return -1;
    if (space != 0 && basis == 1) {   // N2curl_k / BDM_k: the full P_k^dim, k = 1..4
        if (order < 1 || order > 4 || (dim != 2 && dim != 3)) return -1;
        return dim == 2 ? (order + 1) * (order + 2) : (order + 1) * (order + 2) * (order + 3) / 2;
    }
    if (space == 0) {
        if (dim == 2 && order >= 1 && order <= 4) return (order + 1) * (order + 2) / 2;
        if (dim == 3 && order >= 1 && order <= 4) return (order + 1) * (order + 2) * (order + 3) / 6;
        return -1;
    }
    if (order < 1 || order > 4) return -1;
    if (dim == 2 && (space == 1 || space == 2)) return order * (order + 2);
    if (dim != 3) return -1;
    if (space == 1) return order * (order + 2) * (order + 3) / 2;
    if (space == 2) return order * (order + 1) * (order + 3) / 2;
    return -1;
}

// ---- Bernstein ------------------------------------------------------------------------
// B_a = p!/a! prod_i lambda_i^{a_i} over the same multi-indices as the Lagrange nodes.  The
// reference mass is exact in closed form: the integral of lambda^g over the reference simplex
// (volume 1/d!) is g! / (|g| + d)!, so int B_a B_b = (p!)^2 / (a! b!) (a + b)! / (2p + d)!.
// All factorials are integers below 2^53 for p <= 4, d <= 3; one rounding at the end.
int build_bernstein(int dim, int p, RefTables* out) {
    std::vector<std::vector<int>> nodes;
    compositions(dim + 1, p, nodes);
    const int n = (int)nodes.size();
    auto fact = [](int k) {
        double f = 1;
        for (int i = 2; i <= k; ++i) f *= i;
        return f;
    };
    out->nloc = n;
    out->ncomp = 1;
    out->R.assign((size_t)n * n, 0.0);
    const double den = fact(2 * p + dim);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double num = fact(p) * fact(p), dab = 1;
            for (int k = 0; k <= dim; ++k) {
                num *= fact(nodes[i][k] + nodes[j][k]);
                dab *= fact(nodes[i][k]) * fact(nodes[j][k]);
            }
            out->R[(size_t)i * n + j] = num / (dab * den);
        }
    return 0;
}

int build_reference(int dim, int space, int order, RefTables* out, int basis) {
    if (n_local(dim, space, order, basis) < 0) return -1;
    out->dim = dim;
    out->space = space;
    out->order = order;
    if (space == 0) {
        if (basis == 1) return build_bernstein(dim, order, out);
        if (basis == 2) return build_lagrange_gll(dim, order, out);
        return build_lagrange(dim, order, out);
    }
    if (basis == 1) return build_second_kind(dim, space == 1, order, out);
    if (dim == 2) return build_vector_2d(space == 1, order, out);
    return build_vector(space == 1, order, out);
}

}  // namespace bras
