// Host FP64 precompute of the kiFMM operators (the one place FP64 is used on the fast path's
// behalf).  Everything is built once per (p, pinv_rtol, svd_rtol, kappa_u) in units of the box
// half-width and cached for the life of the process; kappa_u = 0 is the Laplace kernel, whose
// one set serves every level, and kappa_u = kappa r_l gives level l's modified Helmholtz set.
//
// Operators (Table 1 of the paper, algebraic kiFMM of Section 2.1), with the box data held as
// check potentials (see fmm_internal.h):
//   UC2E = pinv(K(uc, ue)), DC2E = pinv(K(dc, de)) on the unit box (truncated SVD);
//   A_c  = K(uc_P, ue_c) * pinv(K(uc_c, ue_c))  U2U, child half-width 1/2 ((1/2) UC2E for Laplace)
//   B_c  = K(dc_c, de_P) * DC2E             D2D
//   T_t  = K(dc_0, ue_{2 t}) * UC2E         VLI for transfer vector t (316 of them; the
//                                           translational symmetry of Section 2.2)
//   T_t ~ Uo C_t Vi^T with Uo, Vi from the SVDs of [T_1 ... T_316] and [T_1; ...; T_316]
//   close: DC2E = (V S^-1)(U^T) kept factored.
// Surfaces: a surface of order p around a box of centre c and half-width r is the grid
// c + alpha r (2 idx/(p-1) - 1), idx in {0..p-1}^3 with an index at 0 or p-1 (lexicographic),
// 6(p-1)^2+2 points (Section 4, global portion); alpha = 1.05 for the upward-equivalent and
// downward-check surfaces, 2.95 for the upward-check and downward-equivalent surfaces.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr double kInv4Pi = 0.079577471545947667884441881686257181;
constexpr double kAlphaInner = 1.05;
constexpr double kAlphaOuter = 2.95;

using Mat = std::vector<double>;  // row-major

int hw_threads() {
    unsigned n = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(n, 32u));
}

template <class F>
void parallel_for(int n, F f) {
    int nt = std::min(hw_threads(), n);
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = t; i < n; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

// C[m x n] = A[m x k] * B[k x n]
Mat matmul(const Mat &a, const Mat &b, int m, int k, int n) {
    Mat c((size_t)m * n, 0.0);
    for (int i = 0; i < m; ++i) {
        double *ci = &c[(size_t)i * n];
        for (int l = 0; l < k; ++l) {
            const double ail = a[(size_t)i * k + l];
            if (ail == 0.0) continue;
            const double *bl = &b[(size_t)l * n];
            for (int j = 0; j < n; ++j) ci[j] += ail * bl[j];
        }
    }
    return c;
}

Mat transpose(const Mat &a, int m, int n) {
    Mat t((size_t)m * n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) t[(size_t)j * m + i] = a[(size_t)i * n + j];
    return t;
}

Mat scaled_surface(const std::vector<double> &grid, double cx, double cy, double cz, double r,
                   double alpha) {
    Mat s(grid.size());
    for (size_t i = 0; i < grid.size() / 3; ++i) {
        s[3 * i] = cx + alpha * r * grid[3 * i];
        s[3 * i + 1] = cy + alpha * r * grid[3 * i + 1];
        s[3 * i + 2] = cz + alpha * r * grid[3 * i + 2];
    }
    return s;
}

// K(x_i, y_j) = 1/(4 pi |x_i - y_j|) (Eq. 2 normalised), with kernel FMM_YUKAWA the modified
// Helmholtz kernel exp(-param |x_i - y_j|) / (4 pi |x_i - y_j|), 0 where the points coincide; an
// m x n matrix.  With FMM_HELMHOLTZ the kernel exp(i param |x_i - y_j|) / (4 pi |x_i - y_j|) is
// complex and the result is its real form [[Re K, -Im K], [Im K, Re K]] (2m x 2n), which maps the
// real vector [Re v; Im v] to [Re Kv; Im Kv].  Products, transposes and pseudo-inverses of real
// forms are the real forms of the complex ones, so every operator below is built unchanged.
Mat kernel_matrix(const Mat &x, const Mat &y, int kernel, double param) {
    const int m = (int)x.size() / 3, n = (int)y.size() / 3;
    const bool cplx = kernel == FMM_HELMHOLTZ;
    const int ld = cplx ? 2 * n : n;
    Mat k((size_t)(cplx ? 2 * m : m) * ld, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double dx = x[3 * i] - y[3 * j], dy = x[3 * i + 1] - y[3 * j + 1],
                   dz = x[3 * i + 2] - y[3 * j + 2];
            double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r > 0.0)) continue;
            if (!cplx) {
                k[(size_t)i * n + j] = kInv4Pi * (kernel == FMM_YUKAWA ? std::exp(-param * r) : 1.0) / r;
                continue;
            }
            const double re = kInv4Pi * std::cos(param * r) / r, im = kInv4Pi * std::sin(param * r) / r;
            k[(size_t)i * ld + j] = re;
            k[(size_t)i * ld + n + j] = -im;
            k[(size_t)(m + i) * ld + j] = im;
            k[(size_t)(m + i) * ld + n + j] = re;
        }
    return k;
}

// One-sided (Hestenes) Jacobi SVD of a square n x n matrix: A = U diag(s) V^T, s descending.
void jacobi_svd(const Mat &a_in, int n, Mat &u, std::vector<double> &s, Mat &v) {
    // work on columns: store A^T rows = A columns for contiguous access
    Mat w = transpose(a_in, n, n);   // w[j*n + i] = A[i][j]
    Mat vt((size_t)n * n, 0.0);      // vt[j*n + i] = V[i][j]
    for (int i = 0; i < n; ++i) vt[(size_t)i * n + i] = 1.0;
    const double tol = 1e-15;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *cp = &w[(size_t)p * n], *cq = &w[(size_t)q * n];
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < n; ++i) {
                    alpha += cp[i] * cp[i];
                    beta += cq[i] * cq[i];
                    gamma += cp[i] * cq[i];
                }
                if (gamma == 0.0) continue;
                double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
                if (!(rel > tol)) continue;
                off = std::max(off, rel);
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < n; ++i) {
                    double x = cp[i], y = cq[i];
                    cp[i] = c * x - sn * y;
                    cq[i] = sn * x + c * y;
                }
                double *vp = &vt[(size_t)p * n], *vq = &vt[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - sn * y;
                    vq[i] = sn * x + c * y;
                }
            }
        }
        if (off <= tol) break;
    }
    std::vector<double> norms(n);
    for (int j = 0; j < n; ++j) {
        double acc = 0;
        for (int i = 0; i < n; ++i) acc += w[(size_t)j * n + i] * w[(size_t)j * n + i];
        norms[j] = std::sqrt(acc);
    }
    std::vector<int> order(n);
    for (int j = 0; j < n; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return norms[a] > norms[b]; });
    u.assign((size_t)n * n, 0.0);
    v.assign((size_t)n * n, 0.0);
    s.assign(n, 0.0);
    for (int jj = 0; jj < n; ++jj) {
        int j = order[jj];
        s[jj] = norms[j];
        for (int i = 0; i < n; ++i) {
            u[(size_t)i * n + jj] = norms[j] > 0 ? w[(size_t)j * n + i] / norms[j] : 0.0;
            v[(size_t)i * n + jj] = vt[(size_t)j * n + i];
        }
    }
}

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix: G = Q diag(l) Q^T, l descending.
void jacobi_eig(const Mat &g_in, int n, Mat &q, std::vector<double> &lam) {
    Mat a = g_in;
    Mat qt((size_t)n * n, 0.0);  // rows are eigenvectors
    for (int i = 0; i < n; ++i) qt[(size_t)i * n + i] = 1.0;
    double scale = 0;
    for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(a[(size_t)i * n + i]));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int r = p + 1; r < n; ++r) off = std::max(off, std::fabs(a[(size_t)p * n + r]));
        if (off <= 1e-17 * scale) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int r = p + 1; r < n; ++r) {
                double apr = a[(size_t)p * n + r];
                if (std::fabs(apr) <= 1e-19 * scale) continue;
                double app = a[(size_t)p * n + p], arr = a[(size_t)r * n + r];
                double theta = (arr - app) / (2.0 * apr);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, r
                    double akp = a[(size_t)k * n + p], akr = a[(size_t)k * n + r];
                    a[(size_t)k * n + p] = c * akp - s * akr;
                    a[(size_t)k * n + r] = s * akp + c * akr;
                }
                for (int k = 0; k < n; ++k) {  // rows p, r
                    double apk = a[(size_t)p * n + k], ark = a[(size_t)r * n + k];
                    a[(size_t)p * n + k] = c * apk - s * ark;
                    a[(size_t)r * n + k] = s * apk + c * ark;
                }
                double *qp = &qt[(size_t)p * n], *qr = &qt[(size_t)r * n];
                for (int k = 0; k < n; ++k) {
                    double x = qp[k], y = qr[k];
                    qp[k] = c * x - s * y;
                    qr[k] = s * x + c * y;
                }
            }
        }
    }
    std::vector<int> order(n);
    for (int j = 0; j < n; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return a[(size_t)x * n + x] > a[(size_t)y * n + y]; });
    q.assign((size_t)n * n, 0.0);
    lam.assign(n, 0.0);
    for (int jj = 0; jj < n; ++jj) {
        int j = order[jj];
        lam[jj] = a[(size_t)j * n + j];
        for (int k = 0; k < n; ++k) q[(size_t)k * n + jj] = qt[(size_t)j * n + k];
    }
}

// Truncated pseudo-inverse factors of a square matrix: pinv = (V S^-1)[:, :r] (U[:, :r])^T.
void pinv_factors(const Mat &a, int n, double rtol, Mat &vsinv, Mat &ut, int &rank) {
    Mat u, v;
    std::vector<double> s;
    jacobi_svd(a, n, u, s, v);
    rank = 0;
    while (rank < n && s[rank] >= rtol * s[0] && s[rank] > 0) ++rank;
    vsinv.assign((size_t)n * rank, 0.0);
    ut.assign((size_t)rank * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < rank; ++j) vsinv[(size_t)i * rank + j] = v[(size_t)i * n + j] / s[j];
    for (int j = 0; j < rank; ++j)
        for (int i = 0; i < n; ++i) ut[(size_t)j * n + i] = u[(size_t)i * n + j];
}

void transfer_vector(int t, int &dx, int &dy, int &dz) {
    int k = 0;
    for (int i = -3; i <= 3; ++i)
        for (int j = -3; j <= 3; ++j)
            for (int l = -3; l <= 3; ++l) {
                if (std::max(std::abs(i), std::max(std::abs(j), std::abs(l))) <= 1) continue;
                if (k == t) {
                    dx = i, dy = j, dz = l;
                    return;
                }
                ++k;
            }
}

int transfer_index_of(int dx, int dy, int dz) {
    int k = 0;
    for (int i = -3; i <= 3; ++i)
        for (int j = -3; j <= 3; ++j)
            for (int l = -3; l <= 3; ++l) {
                if (std::max(std::abs(i), std::max(std::abs(j), std::abs(l))) <= 1) continue;
                if (i == dx && j == dy && l == dz) return k;
                ++k;
            }
    return -1;
}

// Operators of one level, up to the choice of the M2L ranks: everything in units of the level's
// box half-width r, where the kernel of a level is (1/r) times the unit-box kernel with
// kappa_u = kappa r (the factor 1/r cancels in every "evaluation o pseudo-inverse" product and
// is applied to the leaf closing by the caller).  For Laplace kappa_u = 0 and one set serves all
// levels.
struct LevelBuild {
    std::unique_ptr<HostOps> h;
    std::vector<Mat> T;                 // the 316 M2L operators
    Mat ql, qr;                         // eigenvectors of the two Gram matrices (descending)
    std::vector<double> ll, lr;         // their eigenvalues
};

// FFT form of the M2L (Section 2.2 names it beside the BLAS form): with the upward-equivalent
// and downward-check surfaces on radius alpha = (p - 1)/(p - 2) half-widths, the grid spacing
// h = 2 alpha / (p - 1) divides the box width 2 (m = p - 2 steps), so every surface point
// difference between a target box and a V-list source at transfer vector t is a lattice vector
// h (d - m t), d in [-(p-1), p-1]^3.  The M2L of t is then the convolution of the source's
// densities (on the p^3 grid, zero off the surface) with K sampled on those vectors, evaluated
// zero-padded to n = 2p points per axis through the discrete Fourier transform.  Unit box
// (half-width 1); for Laplace the transforms serve every level (homogeneity: the M2L of check
// potentials, K(dc, ue) UC2E, is level-invariant).
double lattice_alpha(int p) { return (double)(p - 1) / (double)(p - 2); }

// Real-to-complex DFT of the sampled kernel of transfer vector (tx, ty, tz): out[(ka n + kb) nh
// + kc] = sum_{a,b,c} g[a][b][c] e^{-2 pi i (a ka + b kb + c kc) / n}, nh = n/2 + 1, as
// (re, im) pairs; separable, in FP64.
void lattice_kernel_transform(int p, int tx, int ty, int tz, int kernel, double kappa_u, double *out) {
    const int n = 2 * p, nh = n / 2 + 1, m = p - 2;
    const double h = 2.0 / (p - 2);
    std::vector<double> g((size_t)n * n * n, 0.0);
    auto diff = [&](int i) { return i < p ? i : i - n; };   // circular index -> lattice difference
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c) {
                const int da = diff(a), db = diff(b), dc = diff(c);
                if (std::abs(da) > p - 1 || std::abs(db) > p - 1 || std::abs(dc) > p - 1) continue;
                const double x[3] = {h * (da - m * tx), h * (db - m * ty), h * (dc - m * tz)}, z[3] = {0, 0, 0};
                if (x[0] == 0 && x[1] == 0 && x[2] == 0) continue;
                g[((size_t)a * n + b) * n + c] = fmm::kernel_matrix(Mat(x, x + 3), Mat(z, z + 3), kernel, kappa_u)[0];
            }
    std::vector<double> cr(n), ci(n);
    for (int k = 0; k < n; ++k) cr[k] = std::cos(2.0 * M_PI * k / n), ci[k] = -std::sin(2.0 * M_PI * k / n);
    // along c (real -> half spectrum), then b, then a (complex)
    std::vector<double> s1((size_t)n * n * nh * 2), s2((size_t)n * n * nh * 2);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int kc = 0; kc < nh; ++kc) {
                double re = 0, im = 0;
                for (int c = 0; c < n; ++c) {
                    const double v = g[((size_t)a * n + b) * n + c];
                    const int w = (c * kc) % n;
                    re += v * cr[w], im += v * ci[w];
                }
                s1[(((size_t)a * n + b) * nh + kc) * 2] = re, s1[(((size_t)a * n + b) * nh + kc) * 2 + 1] = im;
            }
    for (int a = 0; a < n; ++a)
        for (int kb = 0; kb < n; ++kb)
            for (int kc = 0; kc < nh; ++kc) {
                double re = 0, im = 0;
                for (int b = 0; b < n; ++b) {
                    const double *v = &s1[(((size_t)a * n + b) * nh + kc) * 2];
                    const int w = (b * kb) % n;
                    re += v[0] * cr[w] - v[1] * ci[w], im += v[0] * ci[w] + v[1] * cr[w];
                }
                s2[(((size_t)a * n + kb) * nh + kc) * 2] = re, s2[(((size_t)a * n + kb) * nh + kc) * 2 + 1] = im;
            }
    for (int ka = 0; ka < n; ++ka)
        for (int kb = 0; kb < n; ++kb)
            for (int kc = 0; kc < nh; ++kc) {
                double re = 0, im = 0;
                for (int a = 0; a < n; ++a) {
                    const double *v = &s2[(((size_t)a * n + kb) * nh + kc) * 2];
                    const int w = (a * ka) % n;
                    re += v[0] * cr[w] - v[1] * ci[w], im += v[0] * ci[w] + v[1] * cr[w];
                }
                out[(((size_t)ka * n + kb) * nh + kc) * 2] = re, out[(((size_t)ka * n + kb) * nh + kc) * 2 + 1] = im;
            }
}

LevelBuild build_level(int p, double pinv_rtol, int kernel, double kappa_u, bool fft) {
    LevelBuild b;
    b.h = std::make_unique<HostOps>();
    HostOps *h = b.h.get();
    h->p = p;
    h->kernel = kernel;
    h->kappa_u = kappa_u;
    const double alpha_in = fft ? lattice_alpha(p) : kAlphaInner;
    h->alpha_inner = alpha_in;
    std::vector<double> grid = surface_grid(p);
    h->npts = (int)grid.size() / 3;
    // ns: the length of a box vector (the surface points, twice that for complex values)
    const int ns = kernel == FMM_HELMHOLTZ ? 2 * h->npts : h->npts;
    h->ns = ns;
    auto kernel_matrix = [&](const Mat &x, const Mat &y, double param) {
        return fmm::kernel_matrix(x, y, kernel, param);
    };
    Mat ue = scaled_surface(grid, 0, 0, 0, 1.0, alpha_in);     // upward equivalent
    Mat uc = scaled_surface(grid, 0, 0, 0, 1.0, kAlphaOuter);   // upward check
    Mat dc = ue;                                                // downward check (the inner radius)
    Mat de = uc;                                                // downward equivalent (2.95)
    h->surf_inner = ue;
    h->surf_outer = uc;

    // check-to-equivalent pseudo-inverses on the unit box, and the child's (below); the three
    // factorisations are independent and run on threads of their own
    Mat uc_vs, uc_ut, dc_vs, dc_ut, ch_vs, ch_ut;
    int r_uc = 0, r_dc = 0, r_ch = 0;
    {
        std::thread t1([&] { pinv_factors(kernel_matrix(uc, ue, kappa_u), ns, pinv_rtol, uc_vs, uc_ut, r_uc); });
        std::thread t2([&] { pinv_factors(kernel_matrix(dc, de, kappa_u), ns, pinv_rtol, dc_vs, dc_ut, r_dc); });
        if (kappa_u > 0.0) pinv_factors(kernel_matrix(uc, ue, 0.5 * kappa_u), ns, pinv_rtol, ch_vs, ch_ut, r_ch);
        t1.join();
        t2.join();
    }
    Mat uc2e = matmul(uc_vs, uc_ut, ns, r_uc, ns);
    Mat dc2e = matmul(dc_vs, dc_ut, ns, r_dc, ns);
    h->rcl = r_dc;
    h->close1 = dc_ut;   // [r_dc x ns]
    h->close2 = dc_vs;   // [ns x r_dc]
    h->rclu = r_uc;
    h->uclose1 = uc_ut;  // [r_uc x ns]
    h->uclose2 = uc_vs;  // [ns x r_uc]

    // A child box of half-width 1/2 sees the kernel K_{kappa_u}(x/2, y/2) = 2 K_{kappa_u/2}(x, y)
    // of its own unit box (for the Helmholtz kernel with the wavenumber in place of kappa), so
    // its pseudo-inverse is (1/2) pinv(K_{kappa_u/2}(uc, ue)); for Laplace that is (1/2) UC2E.
    Mat child_uc2e = kappa_u > 0.0 ? matmul(ch_vs, ch_ut, ns, r_ch, ns) : uc2e;
    for (auto &x : child_uc2e) x *= 0.5;

    // U2U and D2D per octant (child half-width 1/2, centre offset +-1/2 per axis, x bit first)
    for (int c = 0; c < 8; ++c) {
        double cx = ((c >> 2) & 1) ? 0.5 : -0.5, cy = ((c >> 1) & 1) ? 0.5 : -0.5,
               cz = (c & 1) ? 0.5 : -0.5;
        Mat child_ue = scaled_surface(grid, cx, cy, cz, 0.5, alpha_in);
        Mat child_dc = child_ue;
        h->up[c] = matmul(kernel_matrix(uc, child_ue, kappa_u), child_uc2e, ns, ns, ns);
        h->down[c] = matmul(kernel_matrix(child_dc, de, kappa_u), dc2e, ns, ns, ns);
    }

    if (fft) {   // the lattice kernel's transforms instead of the compressed operators
        const int n = 2 * p, nf = n * n * (n / 2 + 1);
        h->fft_n = n;
        h->fft_ghat.assign((size_t)kNumTransfer * nf * 2, 0.0);
        parallel_for(kNumTransfer, [&](int t) {
            int dx, dy, dz;
            transfer_vector(t, dx, dy, dz);
            lattice_kernel_transform(p, dx, dy, dz, kernel, kappa_u, &h->fft_ghat[(size_t)t * nf * 2]);
        });
        return b;
    }
    // M2L operators T_t = K(dc_0, ue_{2t}) UC2E
    b.T.resize(kNumTransfer);
    parallel_for(kNumTransfer, [&](int t) {
        int dx, dy, dz;
        transfer_vector(t, dx, dy, dz);
        Mat src = scaled_surface(grid, 2.0 * dx, 2.0 * dy, 2.0 * dz, 1.0, alpha_in);
        b.T[t] = matmul(kernel_matrix(dc, src, kappa_u), uc2e, ns, ns, ns);
    });
    // Gram matrices of the fat [T_1 .. T_316] (left) and tall [T_1; ..; T_316] (right) stacks
    int nt = hw_threads();
    std::vector<Mat> gl(nt, Mat((size_t)ns * ns, 0.0)), gr(nt, Mat((size_t)ns * ns, 0.0));
    parallel_for(nt, [&](int w) {
        for (int t = w; t < kNumTransfer; t += nt) {
            const Mat &a = b.T[t];
            Mat at = transpose(a, ns, ns);
            Mat l = matmul(a, at, ns, ns, ns), r = matmul(at, a, ns, ns, ns);
            for (size_t i = 0; i < l.size(); ++i) {
                gl[w][i] += l[i];
                gr[w][i] += r[i];
            }
        }
    });
    for (int w = 1; w < nt; ++w)
        for (size_t i = 0; i < gl[0].size(); ++i) {
            gl[0][i] += gl[w][i];
            gr[0][i] += gr[w][i];
        }
    std::thread te([&] { jacobi_eig(gl[0], ns, b.ql, b.ll); });
    jacobi_eig(gr[0], ns, b.qr, b.lr);
    te.join();
    return b;
}

// sigma_i >= svd_rtol * sigma_1  <=>  lambda_i >= svd_rtol^2 * lambda_1
int rank_of(const std::vector<double> &l, double svd_rtol) {
    const int n = (int)l.size();
    int k = 0;
    while (k < n && l[k] > 0 && l[k] >= svd_rtol * svd_rtol * l[0]) ++k;
    return std::max(k, 1);
}

// The compressed M2L at ranks (kin, kout) and the adjoint operators.
std::unique_ptr<HostOps> finish_level(LevelBuild &b, int kin, int kout) {
    HostOps *h = b.h.get();
    const int ns = h->ns;
    if (h->fft_n) {   // FFT M2L: no compressed operators; the surface operators' transposes as below
        h->kin = h->kout = 0;
        for (int c = 0; c < 8; ++c) {
            h->a_up[c] = transpose(h->down[c], ns, ns);
            h->a_down[c] = transpose(h->up[c], ns, ns);
        }
        h->a_close1 = transpose(h->close2, ns, h->rcl);
        h->a_close2 = transpose(h->close1, h->rcl, ns);
        return std::move(b.h);
    }
    h->kout = kout;
    h->kin = kin;
    Mat uo((size_t)ns * kout), vi((size_t)ns * kin);
    for (int i = 0; i < ns; ++i) {
        for (int j = 0; j < kout; ++j) uo[(size_t)i * kout + j] = b.ql[(size_t)i * ns + j];
        for (int j = 0; j < kin; ++j) vi[(size_t)i * kin + j] = b.qr[(size_t)i * ns + j];
    }
    h->decompress = uo;                       // [ns x kout]
    h->compress = transpose(vi, ns, kin);     // [kin x ns]
    Mat uot = transpose(uo, ns, kout);
    h->stencil.assign((size_t)kNumTransfer * kout * kin, 0.0);
    parallel_for(kNumTransfer, [&](int t) {
        Mat tv = matmul(b.T[t], vi, ns, ns, kin);          // ns x kin
        Mat c = matmul(uot, tv, kout, ns, kin);            // kout x kin
        std::copy(c.begin(), c.end(), h->stencil.begin() + (size_t)t * kout * kin);
    });
    b.T.clear();

    // adjoint operators: transposes, with the stencil re-indexed by the opposite vector
    for (int c = 0; c < 8; ++c) {
        h->a_up[c] = transpose(h->down[c], ns, ns);   // children gather of D2D^T
        h->a_down[c] = transpose(h->up[c], ns, ns);   // parent gather of U2U^T
    }
    h->a_compress = uot;                              // [kout x ns]
    h->a_decompress = vi;                             // [ns x kin]
    h->a_stencil.assign((size_t)kNumTransfer * kin * kout, 0.0);
    for (int t = 0; t < kNumTransfer; ++t) {
        int dx, dy, dz;
        transfer_vector(t, dx, dy, dz);
        int tn = transfer_index_of(-dx, -dy, -dz);
        const double *c = &h->stencil[(size_t)tn * kout * kin];
        double *o = &h->a_stencil[(size_t)t * kin * kout];
        for (int i = 0; i < kout; ++i)
            for (int j = 0; j < kin; ++j) o[(size_t)j * kout + i] = c[(size_t)i * kin + j];
    }
    h->a_close1 = transpose(h->close2, ns, h->rcl);   // [r_dc x ns] = (V S^-1)^T
    h->a_close2 = transpose(h->close1, h->rcl, ns);   // [ns x r_dc] = U
    return std::move(b.h);
}

}  // namespace

std::vector<double> surface_grid(int p) {
    std::vector<double> g;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                bool on = i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1;
                if (!on) continue;
                g.push_back(2.0 * i / (p - 1) - 1.0);
                g.push_back(2.0 * j / (p - 1) - 1.0);
                g.push_back(2.0 * k / (p - 1) - 1.0);
            }
    return g;
}

std::vector<const HostOps *> host_operator_levels(int p, double pinv_rtol, double svd_rtol, int kernel,
                                                  const std::vector<double> &kappa_u, std::string *err, bool fft) {
    static std::mutex mu;
    static std::map<std::tuple<int, double, double, int, std::vector<double>, bool>,
                    std::vector<std::unique_ptr<HostOps>>>
        cache;
    std::lock_guard<std::mutex> lock(mu);
    std::vector<double> key_k = kappa_u;
    for (auto &k : key_k) k = kernel == FMM_LAPLACE ? 0.0 : std::max(k, 0.0);
    auto key = std::make_tuple(p, pinv_rtol, svd_rtol, kernel, key_k, fft);
    auto it = cache.find(key);
    if (it == cache.end()) {
        // distinct kappa_u values only; the M2L ranks are the largest any of them needs, so that
        // every level's contractions have one shape
        std::vector<double> uniq = key_k;
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        std::vector<LevelBuild> lb;
        int kin = 1, kout = 1;
        for (double k : uniq) {
            lb.push_back(build_level(p, pinv_rtol, kernel, k, fft));
            if (fft) continue;
            kin = std::max(kin, rank_of(lb.back().lr, svd_rtol));
            kout = std::max(kout, rank_of(lb.back().ll, svd_rtol));
        }
        std::vector<std::unique_ptr<HostOps>> built;
        for (auto &b : lb) built.push_back(finish_level(b, kin, kout));
        it = cache.emplace(key, std::move(built)).first;
    }
    std::vector<const HostOps *> out;
    for (double k : key_k)
        for (const auto &h : it->second)
            if (h->kappa_u == k) {
                out.push_back(h.get());
                break;
            }
    if (out.size() != key_k.size()) {
        if (err) *err = "operator cache lookup failed";
        return {};
    }
    return out;
}

const HostOps *host_operators(int p, double pinv_rtol, double svd_rtol, std::string *err) {
    auto v = host_operator_levels(p, pinv_rtol, svd_rtol, FMM_LAPLACE, {0.0}, err, false);
    return v.empty() ? nullptr : v[0];
}

}  // namespace fmm
