// Plain, slow FP64 CPU oracle for the block multishift RHMC path of
// de Forcrand & Keegan, "Rational Hybrid Monte Carlo with Block Solvers and
// Multiple Pseudofermions" (arXiv:1808.01829).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links
// or calls this file; only the tests, the smoke check and the benchmark's CPU
// baseline leg do.  It shares no code with the CUDA path.
//
// What it computes, each piece citing the passage it follows:
//  * the even-odd preconditioned unimproved staggered operator of Sec. IV
//    (A = M^dagger M restricted to even sites), in the normalisation
//    M = 2m + D, (D psi)(x) = sum_mu eta_mu(x) [U_mu(x) psi(x+mu)
//    - U_mu(x-mu)^dagger psi(x-mu)], eta_mu(x) = (-1)^(x_0+..+x_{mu-1}),
//    antiperiodic in t when bc_t = -1 (the paper is silent on the
//    normalisation and phases; this is the reading recorded in the design
//    notes).  A = 4 m^2 - D_eo D_oe.
//  * thin QR of a tall block (Sec. III, the qr() of Algorithm 1), by
//    Gram-Schmidt with one re-orthogonalisation pass, R with positive real
//    diagonal;
//  * SBCGrQ, Algorithm 1, step by step in the paper's order and notation;
//  * scalar multishift CG (SCG, Sec. III) for one right-hand side, derived
//    from the CG three-term relation (the n_pf = 1 special case of Alg. 1);
//  * the pseudofermion action S_f = sum_i phi_i^dagger R(A) phi_i with R the
//    partial-fraction rational approximation, Eq. (RA), and its derivative
//    with respect to the links, Eq. (force): G = dS/dRe U + i dS/dIm U.
//
// All complex arrays cross the C interface as interleaved (re, im) doubles.
// Field layout [V/2][3][n]; gauge layout [site][mu][3][3], site = lex index
// x + Lx*(y + Ly*(z + Lz*t)); a site's rank among its parity is lex/2.
//
// Parity of the functions with paper passages that fix them is pinned by the
// tests: free-field spectrum in closed form, hermiticity, positivity, gauge
// covariance, n=1 block solver == scalar CG, dense brute-force solves and
// central finite differences of the action (the latter two against an
// independent numpy implementation).

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cd;

namespace {

struct Lat {
  int L[4];
  double mass;
  int bc_t;
  long V, Vh;
};

bool make_lat(const int *dims, double mass, int bc_t, Lat &l) {
  l.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || dims[mu] % 2) return false;
    l.L[mu] = dims[mu];
    l.V *= dims[mu];
  }
  l.Vh = l.V / 2;
  l.mass = mass;
  l.bc_t = (bc_t == 1) ? 1 : -1;
  return true;
}

inline void coords(const Lat &l, long lex, int x[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    x[mu] = (int)(lex % l.L[mu]);
    lex /= l.L[mu];
  }
}

inline long lexof(const Lat &l, const int x[4]) {
  return x[0] + (long)l.L[0] * (x[1] + (long)l.L[1] * (x[2] + (long)l.L[2] * x[3]));
}

inline int parity(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

// Staggered phase eta_mu(x) = (-1)^(sum_{nu<mu} x_nu).
inline double eta(int mu, const int x[4]) {
  int s = 0;
  for (int nu = 0; nu < mu; ++nu) s += x[nu];
  return (s & 1) ? -1.0 : 1.0;
}

// Boundary sign of the link U_mu(x): -1 on t-links that wrap t = Lt-1 -> 0
// when the temporal boundary condition is antiperiodic.
inline double bsign(const Lat &l, int mu, const int x[4]) {
  return (mu == 3 && x[3] == l.L[3] - 1 && l.bc_t == -1) ? -1.0 : 1.0;
}

// Coordinates of the site with parity p and parity rank h.
inline void site_of(const Lat &l, int p, long h, int x[4]) {
  coords(l, 2 * h, x);
  if (parity(x) != p) coords(l, 2 * h + 1, x);
}

inline void step(const Lat &l, const int x[4], int mu, int dir, int y[4]) {
  for (int nu = 0; nu < 4; ++nu) y[nu] = x[nu];
  y[mu] = (x[mu] + dir + l.L[mu]) % l.L[mu];
}

inline const cd *link(const cd *U, long lex, int mu) { return U + (lex * 4 + mu) * 9; }

// out(x) = D psi restricted to sites x of parity out_par (so psi lives on the
// other parity): sum_mu eta_mu(x) [ b_mu(x) U_mu(x) psi(x+mu)
//                                  - b_mu(x-mu) U_mu(x-mu)^dagger psi(x-mu) ].
void hop_site(const Lat &l, const cd *U, const cd *in, int n, int out_par, long h, cd *out_site) {
  int x[4], y[4];
  site_of(l, out_par, h, x);
  for (int k = 0; k < 3 * n; ++k) out_site[k] = 0.0;
  for (int mu = 0; mu < 4; ++mu) {
    const double e = eta(mu, x);
    // forward neighbour
    step(l, x, mu, +1, y);
    {
      const cd *u = link(U, lexof(l, x), mu);
      const double s = e * bsign(l, mu, x);
      const cd *v = in + (lexof(l, y) / 2) * 3 * n;
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < n; ++j) {
          cd acc = 0.0;
          for (int b = 0; b < 3; ++b) acc += u[a * 3 + b] * v[b * n + j];
          out_site[a * n + j] += s * acc;
        }
    }
    // backward neighbour
    step(l, x, mu, -1, y);
    {
      const cd *u = link(U, lexof(l, y), mu);
      const double s = e * bsign(l, mu, y);
      const cd *v = in + (lexof(l, y) / 2) * 3 * n;
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < n; ++j) {
          cd acc = 0.0;
          for (int b = 0; b < 3; ++b) acc += std::conj(u[b * 3 + a]) * v[b * n + j];
          out_site[a * n + j] -= s * acc;
        }
    }
  }
}

void hop(const Lat &l, const cd *U, const cd *in, cd *out, int n, int out_par) {
#pragma omp parallel for schedule(static)
  for (long h = 0; h < l.Vh; ++h) hop_site(l, U, in, n, out_par, h, out + h * 3 * n);
}

// Y = (A + sigma) X on even sites, A = 4 m^2 - D_eo D_oe.
void apply_A(const Lat &l, const cd *U, const cd *X, cd *Y, int n, double sigma, std::vector<cd> &tmp) {
  const long len = l.Vh * 3 * n;
  tmp.resize(len);
  hop(l, U, X, tmp.data(), n, 1);
  hop(l, U, tmp.data(), Y, n, 0);
  const double c = 4.0 * l.mass * l.mass + sigma;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < len; ++k) Y[k] = c * X[k] - Y[k];
}

// ---------------------------------------------------------------- small n x n
typedef std::vector<cd> Mat;  // row-major n x n

Mat eye(int n) {
  Mat m(n * n, 0.0);
  for (int i = 0; i < n; ++i) m[i * n + i] = 1.0;
  return m;
}
Mat mul(const Mat &a, const Mat &b, int n) {
  Mat c(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j) c[i * n + j] += a[i * n + k] * b[k * n + j];
  return c;
}
Mat adj(const Mat &a, int n) {
  Mat c(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) c[i * n + j] = std::conj(a[j * n + i]);
  return c;
}
Mat add(const Mat &a, const Mat &b, int n, double sb = 1.0) {
  Mat c(n * n);
  for (int k = 0; k < n * n; ++k) c[k] = a[k] + sb * b[k];
  return c;
}
Mat scale(const Mat &a, double s, int n) {
  Mat c(n * n);
  for (int k = 0; k < n * n; ++k) c[k] = s * a[k];
  return c;
}
// Inverse by Gauss-Jordan elimination with partial pivoting; ok=false if singular.
Mat inv(const Mat &a, int n, bool &ok) {
  Mat m = a, r = eye(n);
  ok = true;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::abs(m[i * n + c]) > std::abs(m[p * n + c])) p = i;
    if (!(std::abs(m[p * n + c]) > 0.0) || !std::isfinite(std::abs(m[p * n + c]))) {
      ok = false;
      return r;
    }
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(m[p * n + j], m[c * n + j]);
        std::swap(r[p * n + j], r[c * n + j]);
      }
    const cd d = 1.0 / m[c * n + c];
    for (int j = 0; j < n; ++j) {
      m[c * n + j] *= d;
      r[c * n + j] *= d;
    }
    for (int i = 0; i < n; ++i)
      if (i != c) {
        const cd f = m[i * n + c];
        if (f == 0.0) continue;
        for (int j = 0; j < n; ++j) {
          m[i * n + j] -= f * m[c * n + j];
          r[i * n + j] -= f * r[c * n + j];
        }
      }
  }
  return r;
}
// Euclidean norm of column j of an n x n matrix.
double colnorm(const Mat &a, int n, int j) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += std::norm(a[i * n + j]);
  return std::sqrt(s);
}

// ------------------------------------------------------- tall blocks L x n
// A "block" is a field [Vh][3][n]: L = 3 Vh rows, n columns.

// C = A^dagger B  (n x n), summed over all rows.
Mat gram(const cd *A, const cd *B, long rows, int n) {
  Mat g(n * n, 0.0);
#pragma omp parallel
  {
    Mat loc(n * n, 0.0);
#pragma omp for schedule(static)
    for (long r = 0; r < rows; ++r)
      for (int i = 0; i < n; ++i) {
        const cd ai = std::conj(A[r * n + i]);
        for (int j = 0; j < n; ++j) loc[i * n + j] += ai * B[r * n + j];
      }
#pragma omp critical
    for (int k = 0; k < n * n; ++k) g[k] += loc[k];
  }
  return g;
}

// Y = C + s * A M   (A, C blocks; M n x n).  Y may alias C but not A.
void block_axpy(cd *Y, const cd *C, double s, const cd *A, const Mat &M, long rows, int n) {
#pragma omp parallel for schedule(static)
  for (long r = 0; r < rows; ++r) {
    cd row[64];
    for (int j = 0; j < n; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < n; ++k) acc += A[r * n + k] * M[k * n + j];
      row[j] = acc;
    }
    for (int j = 0; j < n; ++j) Y[r * n + j] = (C ? C[r * n + j] : cd(0.0)) + s * row[j];
  }
}

// Thin QR: B = Q R, Q^dagger Q = 1, R upper triangular with positive real
// diagonal.  Classical Gram-Schmidt applied twice per column.  Returns false
// if a column is (numerically) linearly dependent on the previous ones.
bool thin_qr(const cd *B, cd *Q, Mat &R, long rows, int n) {
  R.assign(n * n, 0.0);
  std::vector<cd> v(rows);
  for (int j = 0; j < n; ++j) {
    for (long r = 0; r < rows; ++r) v[r] = B[r * n + j];
    double norm0 = 0.0;
    for (long r = 0; r < rows; ++r) norm0 += std::norm(v[r]);
    norm0 = std::sqrt(norm0);
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        cd c = 0.0;
        for (long r = 0; r < rows; ++r) c += std::conj(Q[r * n + i]) * v[r];
        R[i * n + j] += c;
        for (long r = 0; r < rows; ++r) v[r] -= c * Q[r * n + i];
      }
    double nv = 0.0;
    for (long r = 0; r < rows; ++r) nv += std::norm(v[r]);
    nv = std::sqrt(nv);
    if (!(nv > 1e-14 * norm0) || !(nv > 0.0) || !std::isfinite(nv)) return false;
    R[j * n + j] = nv;
    for (long r = 0; r < rows; ++r) Q[r * n + j] = v[r] / nv;
  }
  return true;
}

thread_local int g_last_iters = 0;

}  // namespace

// =================================================================== C API
extern "C" {

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// out = D in on sites of parity out_par (0 even, 1 odd).
int orc_hop(const int *dims, int bc_t, const double *U, const double *in, double *out, int n, int out_par) {
  Lat l;
  if (!make_lat(dims, 0.0, bc_t, l) || n <= 0 || n > 64) return 1;
  hop(l, (const cd *)U, (const cd *)in, (cd *)out, n, out_par ? 1 : 0);
  return 0;
}

// Y = (A + sigma) X on even sites.
int orc_apply_A(const int *dims, double mass, int bc_t, const double *U, const double *X, double *Y, int n,
                double sigma) {
  Lat l;
  if (!make_lat(dims, mass, bc_t, l) || n <= 0 || n > 64) return 1;
  std::vector<cd> tmp;
  apply_A(l, (const cd *)U, (const cd *)X, (cd *)Y, n, sigma, tmp);
  return 0;
}

// (A + sigma) X evaluated only at the listed even-site ranks; Y is
// [nsites][3][n].  Each value is computed locally from X, so this works at
// any lattice size without forming a full field.
int orc_apply_A_at(const int *dims, double mass, int bc_t, const double *Uv, const double *Xv, double *Yv, int n,
                   double sigma, const long *sites, long nsites) {
  Lat l;
  if (!make_lat(dims, mass, bc_t, l) || n <= 0 || n > 64) return 1;
  const cd *U = (const cd *)Uv, *X = (const cd *)Xv;
  cd *Y = (cd *)Yv;
  const double c = 4.0 * l.mass * l.mass + sigma;
#pragma omp parallel for schedule(dynamic)
  for (long k = 0; k < nsites; ++k) {
    const long h = sites[k];
    int x[4], y[4], z[4];
    site_of(l, 0, h, x);
    std::vector<cd> acc(3 * n, 0.0), ynb(3 * n);
    // D_eo (D_oe X)(x): the hop to x needs (D_oe X) at the 8 odd neighbours.
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = -1; dir <= 1; dir += 2) {
        step(l, x, mu, dir, y);
        hop_site(l, U, X, n, 1, lexof(l, y) / 2, ynb.data());
        const double e = eta(mu, x);
        if (dir > 0) {
          const cd *u = link(U, lexof(l, x), mu);
          const double s = e * bsign(l, mu, x);
          for (int a = 0; a < 3; ++a)
            for (int j = 0; j < n; ++j) {
              cd t = 0.0;
              for (int b = 0; b < 3; ++b) t += u[a * 3 + b] * ynb[b * n + j];
              acc[a * n + j] += s * t;
            }
        } else {
          for (int nu = 0; nu < 4; ++nu) z[nu] = y[nu];
          const cd *u = link(U, lexof(l, z), mu);
          const double s = e * bsign(l, mu, z);
          for (int a = 0; a < 3; ++a)
            for (int j = 0; j < n; ++j) {
              cd t = 0.0;
              for (int b = 0; b < 3; ++b) t += std::conj(u[b * 3 + a]) * ynb[b * n + j];
              acc[a * n + j] -= s * t;
            }
        }
      }
    for (int q = 0; q < 3 * n; ++q) Y[k * 3 * n + q] = c * X[h * 3 * n + q] - acc[q];
  }
  return 0;
}

// Thin QR of a block B (rows x n): Q (rows x n), R (n x n).  1 on breakdown.
int orc_thin_qr(const double *B, double *Q, double *R, long rows, int n) {
  Mat r;
  if (!thin_qr((const cd *)B, (cd *)Q, r, rows, n)) return 3;
  std::memcpy(R, r.data(), sizeof(cd) * n * n);
  return 0;
}

// SBCGrQ, Algorithm 1: solve (A + sigma_s) X^(s) = B for all shifts at once.
//   B        [Vh][3][n]            right-hand-side block
//   shifts   [nshift], ascending; shifts[0] = sigma_0 drives the Krylov space
//   X        [nshift][Vh][3][n]    output
//   tol      stopping threshold on every column's relative residual,
//            base and shifted (the stopping rule of Alg. 1 read column-wise,
//            as ||delta e_j|| / ||delta_0 e_j||, see the design notes)
//   tol_shift  a shift stops being updated once all its columns are below
//            this (the freezing rule of Sec. III); <=0 means tol
//   fixed_iters > 0: run exactly that many iterations, no stopping/freezing
//   resid    optional [max_iter+1]: max_j base relative residual per iteration
// Returns 0 converged, 2 not converged within max_iter, 3 breakdown,
// 1 bad arguments.  *iters_out gets the number of iterations done.
int orc_sbcgrq(const int *dims, double mass, int bc_t, const double *Uv, const double *Bv, int n, int nshift,
               const double *shifts, double *Xv, double tol, double tol_shift, int max_iter, int fixed_iters,
               int *iters_out, double *resid) {
  Lat l;
  if (!make_lat(dims, mass, bc_t, l) || n <= 0 || n > 64 || nshift <= 0) return 1;
  for (int s = 1; s < nshift; ++s)
    if (!(shifts[s] >= shifts[s - 1])) return 1;
  if (tol_shift <= 0) tol_shift = tol;
  const cd *U = (const cd *)Uv, *B = (const cd *)Bv;
  cd *X = (cd *)Xv;
  const long rows = l.Vh * 3, len = rows * n;
  const double s0 = shifts[0];
  std::vector<cd> Q(len), P(len * nshift), AP(len), W(len), tmp;
  // initialisation: X = 0, {Q_0, delta_0} = qr(B), P^(s) = Q_0
  std::fill(X, X + len * nshift, cd(0.0));
  Mat delta;
  if (!thin_qr(B, Q.data(), delta, rows, n)) return 3;
  for (int s = 0; s < nshift; ++s) std::copy(Q.begin(), Q.end(), P.begin() + s * len);
  std::vector<double> d0(n);
  for (int j = 0; j < n; ++j) d0[j] = colnorm(delta, n, j);
  // initial coefficients: rho_0 = delta_0, alpha_0 = alpha^(s)_0 = beta^(s)_0 = 1
  Mat rho = delta, alpha = eye(n);
  std::vector<Mat> alpha_s(nshift, eye(n)), beta_s(nshift, eye(n));
  std::vector<char> active(nshift, 1);
  if (resid) resid[0] = 1.0;
  int k = 0, status = 2;
  const int kmax = fixed_iters > 0 ? fixed_iters : max_iter;
  while (k < kmax) {
    ++k;
    cd *P0 = P.data();
    // alpha_k = (P^dagger (A + sigma_0) P)^-1
    apply_A(l, U, P0, AP.data(), n, s0, tmp);
    bool ok;
    Mat alpha_k = inv(gram(P0, AP.data(), rows, n), n, ok);
    if (!ok) { status = 3; break; }
    // block QR: {Q_k, rho_k} = qr(Q_{k-1} - (A + sigma_0) P alpha_k)
    block_axpy(W.data(), Q.data(), -1.0, AP.data(), alpha_k, rows, n);
    Mat rho_k;
    if (!thin_qr(W.data(), Q.data(), rho_k, rows, n)) { status = 3; break; }
    // base solution: X^(0) += P alpha_k delta_{k-1}
    block_axpy(X, X, 1.0, P0, mul(alpha_k, delta, n), rows, n);
    // base search block: P^(0) = Q_k + P rho_k^dagger
    block_axpy(P0, nullptr, 1.0, P0, adj(rho_k, n), rows, n);  // P0 <- P0 rho^dag (row-wise, in place safe)
    for (long q = 0; q < len; ++q) P0[q] += Q[q];
    // residual factor: delta_k = rho_k delta_{k-1}
    Mat delta_k = mul(rho_k, delta, n);
    // the shifted systems
    Mat coupling = mul(mul(alpha_k, rho, n), (inv(alpha, n, ok)), n);  // alpha_k rho_{k-1} alpha_{k-1}^-1
    if (!ok) { status = 3; break; }
    bool all_done = true;
    double base_res = 0.0;
    for (int j = 0; j < n; ++j) base_res = std::max(base_res, colnorm(delta_k, n, j) / d0[j]);
    for (int s = 1; s < nshift; ++s) {
      if (!active[s]) continue;
      // beta^(s)_k = (1 + (sigma_s - sigma_0) alpha_k + coupling (1 - beta^(s)_{k-1}) rho_{k-1}^dagger)^-1
      Mat t = add(eye(n), scale(alpha_k, shifts[s] - s0, n), n);
      t = add(t, mul(mul(coupling, add(eye(n), beta_s[s], n, -1.0), n), adj(rho, n), n), n);
      Mat beta_k = inv(t, n, ok);
      if (!ok) { status = 3; break; }
      // alpha^(s)_k = beta^(s)_k coupling alpha^(s)_{k-1}
      Mat alpha_sk = mul(mul(beta_k, coupling, n), alpha_s[s], n);
      cd *Ps = P.data() + s * len;
      cd *Xs = X + s * len;
      // shifted solution: X^(s) += P^(s) alpha^(s)_k
      block_axpy(Xs, Xs, 1.0, Ps, alpha_sk, rows, n);
      // shifted search block: P^(s) = Q_k + P^(s) beta^(s)_k rho_k^dagger
      block_axpy(Ps, nullptr, 1.0, Ps, mul(beta_k, adj(rho_k, n), n), rows, n);
      for (long q = 0; q < len; ++q) Ps[q] += Q[q];
      beta_s[s] = beta_k;
      alpha_s[s] = alpha_sk;
      // shifted residual R^(s) = Q_k delta^(s)_k, delta^(s)_k = rho_k alpha_k^-1 alpha^(s)_k (Sec. III)
      Mat dsk = mul(mul(rho_k, inv(alpha_k, n, ok), n), alpha_sk, n);
      double res = 0.0;
      for (int j = 0; j < n; ++j) res = std::max(res, colnorm(dsk, n, j) / d0[j]);
      if (fixed_iters <= 0 && res < tol_shift) active[s] = 0;
      if (active[s]) all_done = false;
    }
    if (status == 3) break;
    alpha = alpha_k;
    rho = rho_k;
    delta = delta_k;
    if (resid) resid[k] = base_res;
    if (fixed_iters <= 0 && base_res < tol && all_done) {
      status = 0;
      break;
    }
  }
  if (fixed_iters > 0 && status == 2 && k == fixed_iters) status = 0;
  if (iters_out) *iters_out = k;
  g_last_iters = k;
  return status;
}

// Scalar multishift CG (SCG, Sec. III) for one right-hand side b [Vh][3]:
// CG on (A + sigma_0) with the shifted residuals kept collinear, r^s = zeta^s r.
// x [nshift][Vh][3].  Stops when every shift's |r^s|/|b| < tol (frozen shifts
// are no longer updated).  Same return codes as orc_sbcgrq.
int orc_scg(const int *dims, double mass, int bc_t, const double *Uv, const double *bv, int nshift,
            const double *shifts, double *xv, double tol, int max_iter, int fixed_iters, int *iters_out) {
  Lat l;
  if (!make_lat(dims, mass, bc_t, l) || nshift <= 0) return 1;
  for (int s = 1; s < nshift; ++s)
    if (!(shifts[s] >= shifts[s - 1])) return 1;
  const cd *U = (const cd *)Uv, *b = (const cd *)bv;
  cd *x = (cd *)xv;
  const long len = l.Vh * 3;
  const double s0 = shifts[0];
  std::vector<cd> r(b, b + len), Ap(len), tmp;
  std::vector<cd> p((size_t)len * nshift);
  for (int s = 0; s < nshift; ++s) std::copy(b, b + len, p.begin() + s * len);
  std::fill(x, x + len * nshift, cd(0.0));
  auto dot = [&](const cd *u, const cd *v) {
    cd acc = 0.0;
    for (long q = 0; q < len; ++q) acc += std::conj(u[q]) * v[q];
    return acc;
  };
  double rr = std::real(dot(r.data(), r.data()));
  const double bb = rr;
  std::vector<double> zeta(nshift, 1.0), zeta_prev(nshift, 1.0);
  std::vector<char> active(nshift, 1);
  double alpha_prev = 1.0, beta_prev = 0.0;
  int k = 0, status = 2;
  const int kmax = fixed_iters > 0 ? fixed_iters : max_iter;
  while (k < kmax) {
    ++k;
    apply_A(l, U, p.data(), Ap.data(), 1, s0, tmp);
    const double pAp = std::real(dot(p.data(), Ap.data()));
    if (!(pAp > 0.0)) { status = 3; break; }
    const double alpha = rr / pAp;
    // shifted coefficients from the CG three-term relation
    std::vector<double> zeta_next(nshift, 1.0);
    for (int s = 1; s < nshift; ++s) {
      if (!active[s]) continue;
      const double ds = shifts[s] - s0;
      zeta_next[s] = zeta[s] * zeta_prev[s] * alpha_prev /
                     (alpha_prev * zeta_prev[s] * (1.0 + ds * alpha) + alpha * beta_prev * (zeta_prev[s] - zeta[s]));
      const double alpha_s = alpha * zeta_next[s] / zeta[s];
      cd *xs = x + s * len, *ps = p.data() + s * len;
      for (long q = 0; q < len; ++q) xs[q] += alpha_s * ps[q];
    }
    for (long q = 0; q < len; ++q) x[q] += alpha * p[q];
    for (long q = 0; q < len; ++q) r[q] -= alpha * Ap[q];
    const double rr_new = std::real(dot(r.data(), r.data()));
    const double beta = rr_new / rr;
    for (long q = 0; q < len; ++q) p[q] = r[q] + beta * p[q];
    bool all_done = true;
    for (int s = 1; s < nshift; ++s) {
      if (!active[s]) continue;
      const double beta_s = beta * (zeta_next[s] / zeta[s]) * (zeta_next[s] / zeta[s]);
      cd *ps = p.data() + s * len;
      for (long q = 0; q < len; ++q) ps[q] = zeta_next[s] * r[q] + beta_s * ps[q];
      zeta_prev[s] = zeta[s];
      zeta[s] = zeta_next[s];
      if (fixed_iters <= 0 && std::abs(zeta[s]) * std::sqrt(rr_new / bb) < tol) active[s] = 0;
      if (active[s]) all_done = false;
    }
    alpha_prev = alpha;
    beta_prev = beta;
    rr = rr_new;
    if (fixed_iters <= 0 && std::sqrt(rr / bb) < tol && all_done) {
      status = 0;
      break;
    }
  }
  if (fixed_iters > 0 && status == 2 && k == fixed_iters) status = 0;
  if (iters_out) *iters_out = k;
  return status;
}

// Pseudofermion action of Eq. (RA) summed over the n columns of Phi, given
// the shifted solutions X^(s) = (A + beta_s)^-1 Phi:
//   S = sum_i [ alpha_0 phi_i^dagger phi_i + sum_s alpha_s phi_i^dagger X^(s) e_i ].
double orc_action(long vh, int n, int nshift, double alpha0, const double *alpha, const double *Phiv,
                  const double *Xv) {
  const cd *Phi = (const cd *)Phiv, *X = (const cd *)Xv;
  const long len = vh * 3 * n;
  double S = 0.0;
  for (long q = 0; q < len; ++q) S += alpha0 * std::norm(Phi[q]);
  for (int s = 0; s < nshift; ++s) {
    cd acc = 0.0;
    for (long q = 0; q < len; ++q) acc += std::conj(Phi[q]) * X[s * len + q];
    S += alpha[s] * std::real(acc);
  }
  return S;
}

// Derivative of the action with respect to the links (Eq. (force) with the
// rational approximation of Eq. (RA)), G_mu(x) = dS/dRe U_mu(x) + i dS/dIm U_mu(x):
//   G_mu(x) = 2 eps(x) eta_mu(x) b_mu(x) sum_{s,i} alpha_s W_si(x) W_si(x+mu)^dagger,
//   W = X^(s) on even sites, W = D_oe X^(s) on odd sites, eps = +1 even / -1 odd.
// X [nshift][Vh][3][n], G [V][4][3][3].
int orc_force(const int *dims, int bc_t, const double *Uv, const double *Xv, int n, int nshift,
              const double *alpha, double *Gv) {
  Lat l;
  if (!make_lat(dims, 0.0, bc_t, l) || n <= 0 || n > 64 || nshift <= 0) return 1;
  const cd *U = (const cd *)Uv, *X = (const cd *)Xv;
  cd *G = (cd *)Gv;
  const long len = l.Vh * 3 * n;
  std::vector<cd> Y((size_t)len * nshift);
  for (int s = 0; s < nshift; ++s) hop(l, U, X + s * len, Y.data() + s * len, n, 1);
#pragma omp parallel for schedule(static)
  for (long lex = 0; lex < l.V; ++lex) {
    int x[4], y[4];
    coords(l, lex, x);
    const int p = parity(x);
    const double eps = p ? -1.0 : 1.0;
    for (int mu = 0; mu < 4; ++mu) {
      step(l, x, mu, +1, y);
      const long hx = lex / 2, hy = lexof(l, y) / 2;
      const double pre = 2.0 * eps * eta(mu, x) * bsign(l, mu, x);
      cd *g = G + (lex * 4 + mu) * 9;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cd acc = 0.0;
          for (int s = 0; s < nshift; ++s) {
            const cd *Wx = (p ? Y.data() : X) + s * len + hx * 3 * n;
            const cd *Wy = (p ? X : Y.data()) + s * len + hy * 3 * n;
            cd t = 0.0;
            for (int i = 0; i < n; ++i) t += Wx[a * n + i] * std::conj(Wy[b * n + i]);
            acc += alpha[s] * t;
          }
          g[a * 3 + b] = pre * acc;
        }
    }
  }
  return 0;
}

// G at the listed links only: link k is (lex = links[2k], mu = links[2k+1]);
// G [nlinks][3][3].  Computed locally from X, for any lattice size.
int orc_force_at(const int *dims, int bc_t, const double *Uv, const double *Xv, int n, int nshift,
                 const double *alpha, const long *links, long nlinks, double *Gv) {
  Lat l;
  if (!make_lat(dims, 0.0, bc_t, l) || n <= 0 || n > 64 || nshift <= 0) return 1;
  const cd *U = (const cd *)Uv, *X = (const cd *)Xv;
  cd *G = (cd *)Gv;
  const long len = l.Vh * 3 * n;
#pragma omp parallel for schedule(dynamic)
  for (long k = 0; k < nlinks; ++k) {
    const long lex = links[2 * k];
    const int mu = (int)links[2 * k + 1];
    int x[4], y[4];
    coords(l, lex, x);
    step(l, x, mu, +1, y);
    const int p = parity(x);
    const double pre = 2.0 * (p ? -1.0 : 1.0) * eta(mu, x) * bsign(l, mu, x);
    std::vector<cd> wo(3 * n);
    cd g[9] = {};
    for (int s = 0; s < nshift; ++s) {
      const cd *Xs = X + s * len;
      // the odd endpoint's W is D_oe X there
      const long odd_lex = p ? lex : lexof(l, y);
      hop_site(l, U, Xs, n, 1, odd_lex / 2, wo.data());
      const cd *Wx = p ? wo.data() : Xs + (lex / 2) * 3 * n;
      const cd *Wy = p ? Xs + (lexof(l, y) / 2) * 3 * n : wo.data();
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cd t = 0.0;
          for (int i = 0; i < n; ++i) t += Wx[a * n + i] * std::conj(Wy[b * n + i]);
          g[a * 3 + b] += alpha[s] * t;
        }
    }
    for (int q = 0; q < 9; ++q) G[k * 9 + q] = pre * g[q];
  }
  return 0;
}

int orc_last_iters(void) { return g_last_iters; }

}  // extern "C"
