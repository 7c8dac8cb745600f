// Plain CPU oracle for the time-dependent MPS simulation of quantum circuits
// (SaiToh, "A Multiprecision Matrix Calculation Library and Its Extension
// Library for a Matrix-Product-State Simulation of Quantum Computing", 2011).
//
// TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark load this library. The product path (the CUDA
// library under paper_1111_3124_gb300/) never links, loads or calls it, and it
// shares no code with it.
//
// What it computes, in the paper's notation (Sec. 3.1):
//   * the state is kept in the Vidal form of Eq. (1): tensors Q_s (here Gamma_s,
//     2 x m_{s-1} x m_s complex entries) and Schmidt vectors V_s (here Lambda_s);
//   * Lambda_s holds the Schmidt coefficients of the cut (0..s)|(s+1..n-1), Eq. (2);
//   * a U(4) gate on qubits (s, s+1) rewrites only Gamma_s, Lambda_s, Gamma_{s+1};
//     the paper defers the details to Vidal (PRL 91, 147902, 2003), which we
//     follow: contract into theta, split by an SVD, keep the leading Schmidt
//     coefficients, divide the outer Lambdas back out;
//   * very small Schmidt coefficients are truncated out (Sec. 3.1, after Eq. 2);
//   * U(8) gates on three consecutive qubits are elementary gates (Sec. 1, Sec. 3.1):
//     one theta over three sites, split by two successive SVDs.
// Readings where the paper is silent:
//   * truncation keeps sigma_j > max(cutoff, m eps) * ||sigma||_2 (m = rows of
//     the Jacobi working matrix, eps the unit roundoff: values at the SVD's
//     resolution are numerically zero), at most chi_max values, at least one,
//     then renormalises the kept values to unit 2-norm;
//   * ties in sigma are broken by column index (stable descending order);
//   * the first site a gate acts on is the most significant bit of the gate's
//     row/column index (fixed by the worked example of Sec. 3.2: CNOT(0,2)
//     with qubit 0 as control);
//   * the SVD is the one-sided Hestenes-Jacobi method with cyclic-by-rows
//     ordering and the complex rotation of Rutishauser / Demmel-Veselic (1992),
//     stopping when every pair satisfies |a_p^H a_q| <= m*eps*||a_p||*||a_q||;
//     columns with ||a_j|| <= m*eps*||A||_F are numerically zero and are not
//     rotated (as LAPACK's zgesvj treats negligible columns).
//
// Two arithmetic modes share the same templated code: IEEE binary64 and
// IEEE binary128 (__float128 on x86_64, long double on aarch64).

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>
#include <algorithm>
#include <new>

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 f128_t;
#elif defined(__aarch64__) && (__LDBL_MANT_DIG__ == 113)
typedef long double f128_t;
#else
#error "no IEEE binary128 type on this platform"
#endif

namespace {

// ---------------------------------------------------------------- scalars ---

template <class R> struct Num;
template <> struct Num<double> {
  static double eps() { return 1.1102230246251565e-16; }  // 2^-53
  static double sqrt_(double x) { return std::sqrt(x); }
};
template <> struct Num<f128_t> {
  static f128_t eps() {  // 2^-113
    f128_t e = 1;
    for (int i = 0; i < 113; ++i) e /= 2;
    return e;
  }
  // Newton's iteration y <- (y + x/y)/2 from the binary64 root: each step
  // doubles the number of correct bits (53 -> 106 -> 113+).
  static f128_t sqrt_(f128_t x) {
    if (!(x > 0)) return 0;
    f128_t y = (f128_t)std::sqrt((double)x);
    if (!(y > 0)) y = 1;
    for (int i = 0; i < 3; ++i) y = (y + x / y) / 2;
    return y;
  }
};

template <class R> struct Cx {
  R re, im;
  Cx() : re(0), im(0) {}
  Cx(R r, R i = 0) : re(r), im(i) {}
};
template <class R> inline Cx<R> operator+(Cx<R> a, Cx<R> b) { return Cx<R>(a.re + b.re, a.im + b.im); }
template <class R> inline Cx<R> operator-(Cx<R> a, Cx<R> b) { return Cx<R>(a.re - b.re, a.im - b.im); }
template <class R> inline Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return Cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> inline Cx<R> operator*(R s, Cx<R> a) { return Cx<R>(s * a.re, s * a.im); }
template <class R> inline Cx<R> conj(Cx<R> a) { return Cx<R>(a.re, -a.im); }
template <class R> inline R abs2(Cx<R> a) { return a.re * a.re + a.im * a.im; }
template <class R> inline R absc(Cx<R> a) { return Num<R>::sqrt_(abs2(a)); }

// ------------------------------------------------------------- dense SVD ---

// One-sided Hestenes-Jacobi SVD of an m x n matrix A (column-major, m >= n).
// On return A's columns are A V (mutually orthogonal), sigma_j = ||(AV)_j||,
// V (n x n, column-major) is unitary. Returns sweeps used, or -1 if the
// 60-sweep limit was hit.
template <class R>
int jacobi_columns(int m, int n, std::vector<Cx<R>>& A, std::vector<Cx<R>>& V,
                   std::vector<R>& sigma) {
  V.assign((size_t)n * n, Cx<R>());
  for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = Cx<R>(1);
  const R tol = Num<R>::eps() * (R)m;
  // Columns with ||a_j|| <= m eps ||A||_F are numerically zero (rounding noise
  // of exact zeros): they take part in no rotation. ||A||_F is invariant.
  R frob = 0;
  for (size_t e = 0; e < A.size(); ++e) frob += abs2(A[e]);
  const R tiny = tol * tol * frob;
  int sweep = 0;
  bool rotated = true;
  while (rotated) {
    if (sweep == 60) return -1;
    rotated = false;
    ++sweep;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        Cx<R>* ap = &A[(size_t)p * m];
        Cx<R>* aq = &A[(size_t)q * m];
        R alpha = 0, beta = 0;
        Cx<R> gamma;
        for (int r = 0; r < m; ++r) {
          alpha += abs2(ap[r]);
          beta += abs2(aq[r]);
          gamma = gamma + conj(ap[r]) * aq[r];
        }
        if (!(alpha > tiny) || !(beta > tiny)) continue;
        R g = absc(gamma);
        if (!(g > tol * Num<R>::sqrt_(alpha) * Num<R>::sqrt_(beta))) continue;
        rotated = true;
        // 2x2 Hermitian [alpha gamma; conj(gamma) beta] = D [alpha g; g beta] D^H
        // with D = diag(1, e^{-i phi}); the real Jacobi rotation of the middle
        // matrix (Golub & Van Loan, sym.schur2) conjugated by D gives
        // J = [c, s e^{i phi}; -s e^{-i phi}, c].
        R zeta = (beta - alpha) / (2 * g);
        R t = 1 / ((zeta >= 0 ? zeta : -zeta) + Num<R>::sqrt_(1 + zeta * zeta));
        if (zeta < 0) t = -t;
        R c = 1 / Num<R>::sqrt_(1 + t * t);
        R s = c * t;
        Cx<R> eip((R)(gamma.re / g), (R)(gamma.im / g));  // e^{i phi}
        Cx<R> s_eip = s * eip;                            // s e^{i phi}
        Cx<R> s_emip = s * conj(eip);                     // s e^{-i phi}
        for (int r = 0; r < m; ++r) {
          Cx<R> x = ap[r], y = aq[r];
          ap[r] = c * x - s_emip * y;
          aq[r] = s_eip * x + c * y;
        }
        Cx<R>* vp = &V[(size_t)p * n];
        Cx<R>* vq = &V[(size_t)q * n];
        for (int r = 0; r < n; ++r) {
          Cx<R> x = vp[r], y = vq[r];
          vp[r] = c * x - s_emip * y;
          vq[r] = s_eip * x + c * y;
        }
      }
    }
  }
  sigma.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    R acc = 0;
    for (int r = 0; r < m; ++r) acc += abs2(A[(size_t)j * m + r]);
    sigma[j] = Num<R>::sqrt_(acc);
  }
  return sweep;
}

// SVD of a general m x n matrix T (row-major): T = X diag(sigma) Y^H with
// r = min(m, n) columns in X (m x r) and Y (n x r), column-major, columns
// normalised where sigma_j > 0. Orientation: Jacobi on the columns of T if
// m >= n, else on the columns of T^H.
template <class R>
int svd_general(int m, int n, const std::vector<Cx<R>>& T, std::vector<R>& sigma,
                std::vector<Cx<R>>& X, std::vector<Cx<R>>& Y) {
  const bool tall = m >= n;
  const int mw = tall ? m : n, nw = tall ? n : m;
  std::vector<Cx<R>> A((size_t)mw * nw), V;
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < n; ++c) {
      if (tall) A[(size_t)c * m + r] = T[(size_t)r * n + c];
      else A[(size_t)r * n + c] = conj(T[(size_t)r * n + c]);
    }
  int sw = jacobi_columns<R>(mw, nw, A, V, sigma);
  // columns of A / sigma are the left vectors of the working matrix
  for (int j = 0; j < nw; ++j) {
    R sj = sigma[j];
    for (int r = 0; r < mw; ++r)
      A[(size_t)j * mw + r] = sj > 0 ? (1 / sj) * A[(size_t)j * mw + r] : Cx<R>();
  }
  if (tall) { X.swap(A); Y.swap(V); }
  else { X.swap(V); Y.swap(A); }  // T^H = A S V^H  =>  T = V S A^H
  return sw;
}

// Descending order of sigma, ties broken by the smaller index first.
template <class R>
std::vector<int> order_desc(const std::vector<R>& s) {
  std::vector<int> p(s.size());
  for (size_t i = 0; i < p.size(); ++i) p[i] = (int)i;
  std::stable_sort(p.begin(), p.end(), [&](int a, int b) { return s[a] > s[b]; });
  return p;
}

struct TruncInfo { int k; double discarded; };

// Truncation of a spectrum: keep sigma_j > cutoff * ||sigma||, at most chi_max
// values, at least one; the kept values, renormalised to unit 2-norm, become
// the new Schmidt vector.
// Values at or below the SVD's resolution, mw * eps * ||sigma|| (mw = rows of
// the Jacobi working matrix), count as zero whatever the cutoff.
template <class R>
TruncInfo truncate(const std::vector<R>& sigma, const std::vector<int>& ord, int chi_max,
                   double cutoff, int mw, std::vector<R>& lam) {
  R total = 0;
  for (R s : sigma) total += s * s;
  R rel = (R)cutoff;
  const R floor_ = Num<R>::eps() * (R)mw;
  if (rel < floor_) rel = floor_;
  R thr = rel * Num<R>::sqrt_(total);
  int k = 0;
  for (int j : ord) if (sigma[j] > thr) ++k;
  if (k > chi_max) k = chi_max;
  if (k < 1) k = 1;
  R kept = 0, dropped = 0;
  for (int c = 0; c < k; ++c) kept += sigma[ord[c]] * sigma[ord[c]];
  for (size_t c = k; c < ord.size(); ++c) dropped += sigma[ord[c]] * sigma[ord[c]];
  lam.resize(k);
  R nk = Num<R>::sqrt_(kept);
  for (int c = 0; c < k; ++c) lam[c] = nk > 0 ? sigma[ord[c]] / nk : (c == 0 ? (R)1 : (R)0);
  TruncInfo ti;
  ti.k = k;
  ti.discarded = total > 0 ? (double)(dropped / total) : 0.0;
  return ti;
}

// ----------------------------------------------------------------- the MPS ---

struct Diag { int k; double discarded; int sweeps; int status; };

class OracleBase {
 public:
  virtual ~OracleBase() {}
  virtual int apply(int site, int k, const double* U) = 0;
  virtual int apply_hl(int site, int k, const double* hi, const double* lo) = 0;
  virtual void amplitude(const unsigned char* bits, double* out) = 0;
  virtual void amplitude_hl(const unsigned char* bits, double* out) = 0;
  virtual void schmidt_hl(int b, double* hi, double* lo) const = 0;
  virtual int expectation(int site, int k, const double* O, double* out) = 0;
  virtual int rdo(const int* qubits, int nq, double* rho) = 0;
  virtual void sample(const double* u, unsigned char* bits) = 0;
  virtual void pauli(const char* p, double* out) = 0;
  virtual int bond(int b) const = 0;
  virtual void schmidt(int b, double* lam) const = 0;
  virtual int set_state(const int* chi, const double* gam, const double* lam) = 0;
  virtual void get_state(int* chi, double* gam, double* lam) const = 0;
  virtual Diag last() const = 0;
  int n, chi_max;
  double cutoff;
};

template <class R>
class OracleMPS : public OracleBase {
 public:
  // bond dims chi_[b+1] for b = -1..n-1 (chi_[0] = chi_[n] = 1)
  std::vector<int> chi_;
  std::vector<std::vector<Cx<R>>> G;  // G[s] = Gamma_s, [i][a][c]
  std::vector<std::vector<R>> L;      // L[b+1] = Lambda_b for b = -1..n-1
  Diag diag_;

  OracleMPS(int n_, int chi_max_, double cutoff_) {
    n = n_; chi_max = chi_max_; cutoff = cutoff_;
    chi_.assign(n + 1, 1);
    G.resize(n);
    L.assign(n + 1, std::vector<R>(1, (R)1));
    for (int s = 0; s < n; ++s) {  // |0...0>: Gamma_s[0] = [[1]], Gamma_s[1] = [[0]]
      G[s].assign(2, Cx<R>());
      G[s][0] = Cx<R>(1);
    }
    diag_ = Diag{1, 0.0, 0, 0};
  }
  int cl(int s) const { return chi_[s]; }      // left bond dim of site s
  int cr(int s) const { return chi_[s + 1]; }  // right bond dim of site s
  const std::vector<R>& lam(int b) const { return L[b + 1]; }
  Cx<R>& g(int s, int i, int a, int c) { return G[s][((size_t)i * cl(s) + a) * cr(s) + c]; }
  Cx<R> gc(int s, int i, int a, int c) const { return G[s][((size_t)i * cl(s) + a) * cr(s) + c]; }

  static Cx<R> in(const Cx<R>* U, int idx) { return U[idx]; }

  // a binary128 (or binary64) value as the double pair hi + lo
  static void split(R x, double* hi, double* lo) {
    const double h = (double)x;
    *hi = h;
    *lo = (double)(x - (R)h);
  }

  // ---- one-site gate: Gamma_s[i] <- sum_k u[i,k] Gamma_s[k]
  void apply1(int s, const Cx<R>* U) {
    const int a_n = cl(s), c_n = cr(s);
    std::vector<Cx<R>> out(G[s].size());
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < a_n; ++a)
        for (int c = 0; c < c_n; ++c) {
          Cx<R> acc;
          for (int k = 0; k < 2; ++k) acc = acc + in(U, i * 2 + k) * gc(s, k, a, c);
          out[((size_t)i * a_n + a) * c_n + c] = acc;
        }
    G[s].swap(out);
    diag_ = Diag{cr(s), 0.0, 0, 0};
  }

  // ---- two-site gate on (s, s+1)
  int apply2(int s, const Cx<R>* U) {
    const int xl = cl(s), xm = cr(s), xr = cr(s + 1);
    const std::vector<R>& ll = lam(s - 1);
    const std::vector<R>& lm = lam(s);
    const std::vector<R>& lr = lam(s + 1);
    // T_kl[a,b] = sum_c Lambda_{s-1}[a] Gamma_s[k,a,c] Lambda_s[c] Gamma_{s+1}[l,c,b] Lambda_{s+1}[b]
    std::vector<Cx<R>> T((size_t)4 * xl * xr);
    for (int k = 0; k < 2; ++k)
      for (int l = 0; l < 2; ++l)
        for (int a = 0; a < xl; ++a)
          for (int b = 0; b < xr; ++b) {
            Cx<R> acc;
            for (int c = 0; c < xm; ++c) acc = acc + (lm[c] * gc(s, k, a, c)) * gc(s + 1, l, c, b);
            T[(((size_t)(k * 2 + l) * xl) + a) * xr + b] = (ll[a] * lr[b]) * acc;
          }
    // theta[(i,a),(j,b)] = sum_{kl} U[(ij),(kl)] T_kl[a,b]; rows i*xl+a, cols j*xr+b
    const int M = 2 * xl, N = 2 * xr;
    std::vector<Cx<R>> th((size_t)M * N);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int a = 0; a < xl; ++a)
          for (int b = 0; b < xr; ++b) {
            Cx<R> acc;
            for (int kl = 0; kl < 4; ++kl)
              acc = acc + in(U, (i * 2 + j) * 4 + kl) * T[((size_t)kl * xl + a) * xr + b];
            th[((size_t)(i * xl + a)) * N + (j * xr + b)] = acc;
          }
    std::vector<R> sigma, newlam;
    std::vector<Cx<R>> X, Y;
    int sw = svd_general<R>(M, N, th, sigma, X, Y);
    if (sw < 0) { diag_ = Diag{0, 0, 60, -4}; return -4; }
    std::vector<int> ord = order_desc(sigma);
    TruncInfo ti = truncate<R>(sigma, ord, chi_max, cutoff, M > N ? M : N, newlam);
    const int kk = ti.k, r = (int)sigma.size();
    // Gamma'_s[i,a,c] = X[(i,a), ord c] / Lambda_{s-1}[a]
    std::vector<Cx<R>> g0((size_t)2 * xl * kk), g1((size_t)2 * kk * xr);
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < xl; ++a)
        for (int c = 0; c < kk; ++c)
          g0[((size_t)i * xl + a) * kk + c] = (1 / ll[a]) * X[(size_t)ord[c] * M + (i * xl + a)];
    // Gamma'_{s+1}[j,c,b] = conj(Y[(j,b), ord c]) / Lambda_{s+1}[b]
    for (int j = 0; j < 2; ++j)
      for (int c = 0; c < kk; ++c)
        for (int b = 0; b < xr; ++b)
          g1[((size_t)j * kk + c) * xr + b] = (1 / lr[b]) * conj(Y[(size_t)ord[c] * N + (j * xr + b)]);
    (void)r;
    G[s].swap(g0);
    G[s + 1].swap(g1);
    L[s + 1] = newlam;
    chi_[s + 1] = kk;
    diag_ = Diag{kk, ti.discarded, sw, 0};
    return 0;
  }

  // ---- three-site gate on (s, s+1, s+2): one theta, two successive splits
  int apply3(int s, const Cx<R>* U) {
    const int xl = cl(s), x1 = cr(s), x2 = cr(s + 1), xr = cr(s + 2);
    const std::vector<R>& ll = lam(s - 1);
    const std::vector<R>& l1 = lam(s);
    const std::vector<R>& l2 = lam(s + 1);
    const std::vector<R>& lr = lam(s + 2);
    // B_{mn}[c,b] = sum_d Gamma_{s+1}[m,c,d] Lambda_{s+1}[d] Gamma_{s+2}[n,d,b] Lambda_{s+2}[b]
    std::vector<Cx<R>> B((size_t)4 * x1 * xr);
    for (int m = 0; m < 2; ++m)
      for (int nn = 0; nn < 2; ++nn)
        for (int c = 0; c < x1; ++c)
          for (int b = 0; b < xr; ++b) {
            Cx<R> acc;
            for (int d = 0; d < x2; ++d) acc = acc + (l2[d] * gc(s + 1, m, c, d)) * gc(s + 2, nn, d, b);
            B[(((size_t)(m * 2 + nn) * x1) + c) * xr + b] = lr[b] * acc;
          }
    // T_{kmn}[a,b] = Lambda_{s-1}[a] sum_c Gamma_s[k,a,c] Lambda_s[c] B_{mn}[c,b]
    std::vector<Cx<R>> T((size_t)8 * xl * xr);
    for (int k = 0; k < 2; ++k)
      for (int mn = 0; mn < 4; ++mn)
        for (int a = 0; a < xl; ++a)
          for (int b = 0; b < xr; ++b) {
            Cx<R> acc;
            for (int c = 0; c < x1; ++c)
              acc = acc + (l1[c] * gc(s, k, a, c)) * B[(((size_t)mn * x1) + c) * xr + b];
            T[(((size_t)(k * 4 + mn) * xl) + a) * xr + b] = ll[a] * acc;
          }
    // theta[(i,a),(j,l,b)] = sum U[(ijl),(kmn)] T_{kmn}[a,b]
    const int M1 = 2 * xl, N1 = 4 * xr;
    std::vector<Cx<R>> th((size_t)M1 * N1);
    for (int i = 0; i < 2; ++i)
      for (int jl = 0; jl < 4; ++jl)
        for (int a = 0; a < xl; ++a)
          for (int b = 0; b < xr; ++b) {
            Cx<R> acc;
            for (int kmn = 0; kmn < 8; ++kmn)
              acc = acc + in(U, (i * 4 + jl) * 8 + kmn) * T[((size_t)kmn * xl + a) * xr + b];
            th[((size_t)(i * xl + a)) * N1 + (jl * xr + b)] = acc;
          }
    std::vector<R> s1, lam1;
    std::vector<Cx<R>> X1, Y1;
    int sw1 = svd_general<R>(M1, N1, th, s1, X1, Y1);
    if (sw1 < 0) { diag_ = Diag{0, 0, 60, -4}; return -4; }
    std::vector<int> o1 = order_desc(s1);
    TruncInfo t1 = truncate<R>(s1, o1, chi_max, cutoff, M1 > N1 ? M1 : N1, lam1);
    const int k1 = t1.k;
    // second matrix: R[c,(j,l,b)] = lam1[c] conj(Y1[(j,l,b), o1 c]), reshaped to rows (j,c), cols (l,b)
    const int M2 = 2 * k1, N2 = 2 * xr;
    std::vector<Cx<R>> th2((size_t)M2 * N2);
    for (int j = 0; j < 2; ++j)
      for (int c = 0; c < k1; ++c)
        for (int l = 0; l < 2; ++l)
          for (int b = 0; b < xr; ++b)
            th2[((size_t)(j * k1 + c)) * N2 + (l * xr + b)] =
                lam1[c] * conj(Y1[(size_t)o1[c] * N1 + ((j * 2 + l) * xr + b)]);
    std::vector<R> s2, lam2;
    std::vector<Cx<R>> X2, Y2;
    int sw2 = svd_general<R>(M2, N2, th2, s2, X2, Y2);
    if (sw2 < 0) { diag_ = Diag{0, 0, 60, -4}; return -4; }
    std::vector<int> o2 = order_desc(s2);
    TruncInfo t2 = truncate<R>(s2, o2, chi_max, cutoff, M2 > N2 ? M2 : N2, lam2);
    const int k2 = t2.k;
    std::vector<Cx<R>> g0((size_t)2 * xl * k1), g1((size_t)2 * k1 * k2), g2((size_t)2 * k2 * xr);
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < xl; ++a)
        for (int c = 0; c < k1; ++c)
          g0[((size_t)i * xl + a) * k1 + c] = (1 / ll[a]) * X1[(size_t)o1[c] * M1 + (i * xl + a)];
    for (int j = 0; j < 2; ++j)
      for (int c = 0; c < k1; ++c)
        for (int d = 0; d < k2; ++d)
          g1[((size_t)j * k1 + c) * k2 + d] = (1 / lam1[c]) * X2[(size_t)o2[d] * M2 + (j * k1 + c)];
    for (int l = 0; l < 2; ++l)
      for (int d = 0; d < k2; ++d)
        for (int b = 0; b < xr; ++b)
          g2[((size_t)l * k2 + d) * xr + b] = (1 / lr[b]) * conj(Y2[(size_t)o2[d] * N2 + (l * xr + b)]);
    G[s].swap(g0);
    G[s + 1].swap(g1);
    G[s + 2].swap(g2);
    L[s + 1] = lam1;
    L[s + 2] = lam2;
    chi_[s + 1] = k1;
    chi_[s + 2] = k2;
    diag_ = Diag{k2, t1.discarded + t2.discarded, sw1 + sw2, 0};
    return 0;
  }

  int apply(int site, int k, const double* U) override { return apply_hl(site, k, U, nullptr); }

  // gate entries hi + lo (lo may be null), formed exactly in R = binary128
  int apply_hl(int site, int k, const double* hi, const double* lo) override {
    const int d = 1 << k;
    std::vector<Cx<R>> u((size_t)d * d);
    for (int e = 0; e < d * d; ++e) {
      R re = (R)hi[2 * e], im = (R)hi[2 * e + 1];
      if (lo) {
        re += (R)lo[2 * e];
        im += (R)lo[2 * e + 1];
      }
      u[e] = Cx<R>(re, im);
    }
    if (k == 1) { apply1(site, u.data()); return 0; }
    if (k == 2) return apply2(site, u.data());
    return apply3(site, u.data());
  }

  // <bits|psi> = Gamma_0[b0] Lambda_0 Gamma_1[b1] Lambda_1 ... Gamma_{n-1}[b_{n-1}]
  void amplitude(const unsigned char* bits, double* out) override {
    const Cx<R> a = amp(bits);
    out[0] = (double)a.re;
    out[1] = (double)a.im;
  }
  // out = (re hi, re lo, im hi, im lo)
  void amplitude_hl(const unsigned char* bits, double* out) override {
    const Cx<R> a = amp(bits);
    split(a.re, out, out + 1);
    split(a.im, out + 2, out + 3);
  }
  Cx<R> amp(const unsigned char* bits) const {
    std::vector<Cx<R>> v(1, Cx<R>(1));
    for (int s = 0; s < n; ++s) {
      const int a_n = cl(s), c_n = cr(s);
      std::vector<Cx<R>> w(c_n);
      for (int c = 0; c < c_n; ++c) {
        Cx<R> acc;
        for (int a = 0; a < a_n; ++a) acc = acc + v[a] * gc(s, bits[s] & 1, a, c);
        w[c] = lam(s)[c] * acc;
      }
      v.swap(w);
    }
    return v[0];
  }

  // A_t[i] = Gamma_t[i] Lambda_t (right Lambda absorbed); the environment
  // E[a,a'] runs over ket index a and bra index a'.
  // ket/bra contraction through one site with physical weights W[i,j]
  // (W = identity for a traced site): E'[c,c'] = sum_{ij} W[i,j] sum_{aa'} A[i,a,c] E[a,a'] conj(A[j,a',c'])
  std::vector<Cx<R>> site_transfer(int s, const std::vector<Cx<R>>& E, const Cx<R>* W) const {
    const int a_n = cl(s), c_n = cr(s);
    std::vector<Cx<R>> out((size_t)c_n * c_n), tmp((size_t)c_n * a_n);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        Cx<R> w = W[i * 2 + j];
        if (w.re == 0 && w.im == 0) continue;
        // tmp[c,a'] = sum_a A[i,a,c] E[a,a']
        for (int c = 0; c < c_n; ++c)
          for (int a2 = 0; a2 < a_n; ++a2) {
            Cx<R> acc;
            for (int a = 0; a < a_n; ++a) acc = acc + (lam(s)[c] * gc(s, i, a, c)) * E[(size_t)a * a_n + a2];
            tmp[(size_t)c * a_n + a2] = acc;
          }
        // out[c,c'] += w * sum_{a'} tmp[c,a'] conj(A[j,a',c'])
        for (int c = 0; c < c_n; ++c)
          for (int c2 = 0; c2 < c_n; ++c2) {
            Cx<R> acc;
            for (int a2 = 0; a2 < a_n; ++a2)
              acc = acc + tmp[(size_t)c * a_n + a2] * conj(lam(s)[c2] * gc(s, j, a2, c2));
            out[(size_t)c * c_n + c2] = out[(size_t)c * c_n + c2] + w * acc;
          }
      }
    return out;
  }

  // <psi|O|psi> / <psi|psi> by full contraction (valid for non-canonical states).
  // O acts on sites site..site+k-1, row index = ket-out bits, col = ket-in bits.
  int expectation(int site, int k, const double* O, double* out) override {
    const int dim = 1 << k;
    // Exact full contraction with the operator block: carry an environment with
    // open (ket-in, bra-out) indices over the k operator sites.
    // E_{xy}[a,a'] where x = ket bits so far, y = bra bits so far.
    std::vector<Cx<R>> E(1, Cx<R>(1));  // 1x1
    const Cx<R> I2[4] = {Cx<R>(1), Cx<R>(), Cx<R>(), Cx<R>(1)};
    for (int s = 0; s < site; ++s) E = site_transfer(s, E, I2);
    // open block
    int width = cl(site);
    std::vector<std::vector<Cx<R>>> blk(1, E);  // index x*cnt + y
    int cnt = 1;
    for (int t = 0; t < k; ++t) {
      const int s = site + t;
      std::vector<std::vector<Cx<R>>> nb((size_t)cnt * 2 * cnt * 2);
      for (int x = 0; x < cnt; ++x)
        for (int y = 0; y < cnt; ++y)
          for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
              Cx<R> W[4] = {Cx<R>(), Cx<R>(), Cx<R>(), Cx<R>()};
              W[i * 2 + j] = Cx<R>(1);
              nb[(size_t)(x * 2 + i) * (cnt * 2) + (y * 2 + j)] = site_transfer(s, blk[(size_t)x * cnt + y], W);
            }
      blk.swap(nb);
      cnt *= 2;
      width = cr(s);
    }
    // contract with O: sum_{x,y} conj-side... ket index x, bra index y:
    // <psi|O|psi> = sum_{x,y} O[y,x] * psi_x conj(psi_y)
    std::vector<Cx<R>> F((size_t)width * width);
    for (int x = 0; x < dim; ++x)
      for (int y = 0; y < dim; ++y) {
        Cx<R> o((R)O[2 * (y * dim + x)], (R)O[2 * (y * dim + x) + 1]);
        for (size_t e = 0; e < F.size(); ++e) F[e] = F[e] + o * blk[(size_t)x * dim + y][e];
      }
    std::vector<Cx<R>> N1 = E;
    for (int t = 0; t < k; ++t) N1 = site_transfer(site + t, N1, I2);
    for (int s = site + k; s < n; ++s) {
      F = site_transfer(s, F, I2);
      N1 = site_transfer(s, N1, I2);
    }
    Cx<R> num = F[0], den = N1[0];
    R d2 = abs2(den);
    Cx<R> q = (1 / d2) * (num * conj(den));
    out[0] = (double)q.re;
    out[1] = (double)q.im;
    return 0;
  }

  // Reduced density operator of the listed qubits (any order, distinct);
  // basis index of rho: the first listed qubit is the most significant bit.
  int rdo(const int* qubits, int nq, double* rho) override {
    std::vector<int> pos(n, -1);
    for (int t = 0; t < nq; ++t) pos[qubits[t]] = t;
    const Cx<R> I2[4] = {Cx<R>(1), Cx<R>(), Cx<R>(), Cx<R>(1)};
    // blocks indexed by (x, y) over open qubits in site order so far
    std::vector<std::vector<Cx<R>>> blk(1, std::vector<Cx<R>>(1, Cx<R>(1)));
    std::vector<int> open_sites;
    int cnt = 1;
    for (int s = 0; s < n; ++s) {
      if (pos[s] < 0) {
        for (auto& b : blk) b = site_transfer(s, b, I2);
        continue;
      }
      std::vector<std::vector<Cx<R>>> nb((size_t)cnt * 2 * cnt * 2);
      for (int x = 0; x < cnt; ++x)
        for (int y = 0; y < cnt; ++y)
          for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
              Cx<R> W[4] = {Cx<R>(), Cx<R>(), Cx<R>(), Cx<R>()};
              W[i * 2 + j] = Cx<R>(1);
              nb[(size_t)(x * 2 + i) * (cnt * 2) + (y * 2 + j)] = site_transfer(s, blk[(size_t)x * cnt + y], W);
            }
      blk.swap(nb);
      cnt *= 2;
      open_sites.push_back(s);
    }
    // trace normalisation
    Cx<R> tr;
    for (int x = 0; x < cnt; ++x) tr = tr + blk[(size_t)x * cnt + x][0];
    R tn = tr.re;
    // map site-ordered bits to requested order
    for (int xs = 0; xs < cnt; ++xs)
      for (int ys = 0; ys < cnt; ++ys) {
        int xr_ = 0, yr_ = 0;
        for (int o = 0; o < nq; ++o) {
          int bitx = (xs >> (nq - 1 - o)) & 1, bity = (ys >> (nq - 1 - o)) & 1;
          int t = pos[open_sites[o]];
          xr_ |= bitx << (nq - 1 - t);
          yr_ |= bity << (nq - 1 - t);
        }
        Cx<R> v = (1 / tn) * blk[(size_t)xs * cnt + ys][0];
        rho[2 * ((size_t)xr_ * cnt + yr_)] = (double)v.re;
        rho[2 * ((size_t)xr_ * cnt + yr_) + 1] = (double)v.im;
      }
    return 0;
  }

  // Right environment through site s: R'[a,a'] = sum_i sum_{c,c'}
  // (Gamma_s[i] Lambda_s)[a,c] R[c,c'] conj((Gamma_s[i] Lambda_s)[a',c']).
  std::vector<Cx<R>> right_transfer(int s, const std::vector<Cx<R>>& Rr) const {
    const int a_n = cl(s), c_n = cr(s);
    std::vector<Cx<R>> out((size_t)a_n * a_n);
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < a_n; ++a)
        for (int a2 = 0; a2 < a_n; ++a2) {
          Cx<R> acc;
          for (int c = 0; c < c_n; ++c)
            for (int c2 = 0; c2 < c_n; ++c2)
              acc = acc + ((lam(s)[c] * gc(s, i, a, c)) * Rr[(size_t)c * c_n + c2]) *
                              conj(lam(s)[c2] * gc(s, i, a2, c2));
          out[(size_t)a * a_n + a2] = out[(size_t)a * a_n + a2] + acc;
        }
    return out;
  }

  // One bit string by sequential conditional sampling of |<b|psi>|^2 /
  // <psi|psi>: qubit s takes 0 when u[s] < p(b_s = 0 | b_0 .. b_{s-1}), else 1.
  // The conditional weights contract the chosen prefix (a row vector v) with
  // the right environments of the rest of the chain.
  void sample(const double* u, unsigned char* bits) override {
    std::vector<std::vector<Cx<R>>> env(n + 1);
    env[n] = std::vector<Cx<R>>(1, Cx<R>(1));
    for (int s = n - 1; s >= 0; --s) env[s] = right_transfer(s, env[s + 1]);
    std::vector<Cx<R>> v(1, Cx<R>(1));
    for (int s = 0; s < n; ++s) {
      const int a_n = cl(s), c_n = cr(s);
      std::vector<Cx<R>> w[2];
      R p[2];
      for (int i = 0; i < 2; ++i) {
        w[i].assign(c_n, Cx<R>());
        for (int c = 0; c < c_n; ++c) {
          Cx<R> acc;
          for (int a = 0; a < a_n; ++a) acc = acc + v[a] * gc(s, i, a, c);
          w[i][c] = lam(s)[c] * acc;
        }
        Cx<R> q;
        for (int c = 0; c < c_n; ++c)
          for (int c2 = 0; c2 < c_n; ++c2) q = q + (w[i][c] * env[s + 1][(size_t)c * c_n + c2]) * conj(w[i][c2]);
        p[i] = q.re;
      }
      const R p0 = p[0] / (p[0] + p[1]);
      const int b = (R)u[s] < p0 ? 0 : 1;
      bits[s] = (unsigned char)b;
      const R inv = 1 / Num<R>::sqrt_(p[b]);
      v.assign(c_n, Cx<R>());
      for (int c = 0; c < c_n; ++c) v[c] = inv * w[b][c];
    }
  }

  // <psi|P|psi> / <psi|psi> for a Pauli string P (one of I, X, Y, Z per
  // qubit): the full transfer contraction with the Pauli matrix as the
  // physical weight at every site.
  void pauli(const char* ps, double* out) override {
    const Cx<R> I2[4] = {Cx<R>(1), Cx<R>(), Cx<R>(), Cx<R>(1)};
    const Cx<R> X2[4] = {Cx<R>(), Cx<R>(1), Cx<R>(1), Cx<R>()};
    const Cx<R> Y2[4] = {Cx<R>(), Cx<R>(0, -1), Cx<R>(0, 1), Cx<R>()};
    const Cx<R> Z2[4] = {Cx<R>(1), Cx<R>(), Cx<R>(), Cx<R>(-1)};
    // W[i,j] weights ket index i against bra index j: <psi|P|psi> = sum P[j,i]... with
    // site_transfer's convention sum_{ij} W[i,j] A_i (x) conj(A_j), W = P^T
    std::vector<Cx<R>> E(1, Cx<R>(1)), N(1, Cx<R>(1));
    for (int s = 0; s < n; ++s) {
      const Cx<R>* P = ps[s] == 'X' ? X2 : ps[s] == 'Y' ? Y2 : ps[s] == 'Z' ? Z2 : I2;
      const Cx<R> W[4] = {P[0], P[2], P[1], P[3]};
      E = site_transfer(s, E, W);
      N = site_transfer(s, N, I2);
    }
    const Cx<R> q = (1 / N[0].re) * E[0];
    out[0] = (double)q.re;
    out[1] = (double)q.im;
  }

  int bond(int b) const override { return chi_[b + 1]; }
  void schmidt(int b, double* out) const override {
    for (int c = 0; c < chi_[b + 1]; ++c) out[c] = (double)L[b + 1][c];
  }
  void schmidt_hl(int b, double* hi, double* lo) const override {
    for (int c = 0; c < chi_[b + 1]; ++c) split(L[b + 1][c], hi + c, lo + c);
  }
  // chi: n+1 bond dims (boundaries 1), gam: concatenated Gamma_s, lam: concatenated Lambda_0..n-2
  int set_state(const int* chi, const double* gam, const double* lamv) override {
    if (chi[0] != 1 || chi[n] != 1) return -1;
    for (int b = 0; b <= n; ++b) if (chi[b] < 1) return -1;  // chi_max caps new bonds only
    chi_.assign(chi, chi + n + 1);
    size_t off = 0;
    for (int s = 0; s < n; ++s) {
      size_t sz = (size_t)2 * chi_[s] * chi_[s + 1];
      G[s].assign(sz, Cx<R>());
      for (size_t e = 0; e < sz; ++e) G[s][e] = Cx<R>((R)gam[2 * (off + e)], (R)gam[2 * (off + e) + 1]);
      off += sz;
    }
    size_t lo = 0;
    L[0] = std::vector<R>(1, (R)1);
    L[n] = std::vector<R>(1, (R)1);
    for (int b = 0; b < n - 1; ++b) {
      L[b + 1].assign(chi_[b + 1], 0);
      for (int c = 0; c < chi_[b + 1]; ++c) L[b + 1][c] = (R)lamv[lo + c];
      lo += chi_[b + 1];
    }
    return 0;
  }
  void get_state(int* chi, double* gam, double* lamv) const override {
    for (int b = 0; b <= n; ++b) chi[b] = chi_[b];
    size_t off = 0;
    for (int s = 0; s < n; ++s) {
      if (gam)
        for (size_t e = 0; e < G[s].size(); ++e) {
          gam[2 * (off + e)] = (double)G[s][e].re;
          gam[2 * (off + e) + 1] = (double)G[s][e].im;
        }
      off += G[s].size();
    }
    size_t lo = 0;
    for (int b = 0; b < n - 1; ++b) {
      if (lamv)
        for (int c = 0; c < chi_[b + 1]; ++c) lamv[lo + c] = (double)L[b + 1][c];
      lo += chi_[b + 1];
    }
  }
  Diag last() const override { return diag_; }
};

}  // namespace

// ------------------------------------------------------------------ C API ---

extern "C" {

// prec: 0 = binary64, 1 = binary128. Returns NULL on bad arguments.
void* oracle_mps_create(int n, int chi_max, double cutoff, int prec) {
  if (n < 1 || chi_max < 1 || !(cutoff >= 0)) return nullptr;
  if (prec == 1) return new (std::nothrow) OracleMPS<f128_t>(n, chi_max, cutoff);
  return new (std::nothrow) OracleMPS<double>(n, chi_max, cutoff);
}
void oracle_mps_destroy(void* h) { delete static_cast<OracleBase*>(h); }

// U: 2^k x 2^k complex128 row-major (re, im interleaved), acting on sites
// site..site+k-1 with the first site as the most significant index bit.
int oracle_mps_apply_gate(void* h, int site, int k, const double* U) {
  OracleBase* m = static_cast<OracleBase*>(h);
  if (!m || !U || k < 1 || k > 3 || site < 0 || site + k > m->n) return -1;
  return m->apply(site, k, U);
}
int oracle_mps_apply_gate_hl(void* h, int site, int k, const double* hi, const double* lo) {
  OracleBase* o = static_cast<OracleBase*>(h);
  if (k < 1 || k > 3 || site < 0 || site + k > o->n) return -1;
  return o->apply_hl(site, k, hi, lo);
}
void oracle_mps_amplitude_hl(void* h, const unsigned char* bits, double* out) {
  static_cast<OracleBase*>(h)->amplitude_hl(bits, out);
}
void oracle_mps_get_schmidt_hl(void* h, int b, double* hi, double* lo) {
  static_cast<OracleBase*>(h)->schmidt_hl(b, hi, lo);
}
void oracle_mps_amplitude(void* h, const unsigned char* bits, double* out) {
  static_cast<OracleBase*>(h)->amplitude(bits, out);
}
int oracle_mps_expectation(void* h, int site, int k, const double* O, double* out) {
  OracleBase* m = static_cast<OracleBase*>(h);
  if (k < 1 || k > 3 || site < 0 || site + k > m->n) return -1;
  return m->expectation(site, k, O, out);
}
int oracle_mps_reduced_density(void* h, const int* qubits, int nq, double* rho) {
  OracleBase* m = static_cast<OracleBase*>(h);
  if (nq < 1 || nq > 10) return -1;
  return m->rdo(qubits, nq, rho);
}
int oracle_mps_bond_dim(void* h, int b) { return static_cast<OracleBase*>(h)->bond(b); }
void oracle_mps_get_schmidt(void* h, int b, double* lam) { static_cast<OracleBase*>(h)->schmidt(b, lam); }
int oracle_mps_set_state(void* h, const int* chi, const double* gam, const double* lam) {
  return static_cast<OracleBase*>(h)->set_state(chi, gam, lam);
}
void oracle_mps_get_state(void* h, int* chi, double* gam, double* lam) {
  static_cast<OracleBase*>(h)->get_state(chi, gam, lam);
}
// k (new bond dim at the last split), discarded weight, Jacobi sweeps, status
void oracle_mps_last_diag(void* h, int* k, double* discarded, int* sweeps, int* status) {
  Diag d = static_cast<OracleBase*>(h)->last();
  *k = d.k; *discarded = d.discarded; *sweeps = d.sweeps; *status = d.status;
}

// One bit string per call: bits[q] for q = 0..n-1 from the uniforms u[0..n-1].
void oracle_mps_sample(void* h, const double* u, unsigned char* bits) {
  static_cast<OracleBase*>(h)->sample(u, bits);
}
// <psi|P|psi>/<psi|psi> for a string of n characters from "IXYZ".
void oracle_mps_pauli(void* h, const char* p, double* out) { static_cast<OracleBase*>(h)->pauli(p, out); }

// Stand-alone SVD of an m x n complex128 matrix T (row-major, interleaved):
// sigma (min(m,n), unsorted, in Jacobi column order), X (m x r, column-major),
// Y (n x r, column-major) with T = X diag(sigma) Y^H. Returns the sweeps used.
int oracle_svd(int prec, int m, int n, const double* T, double* sigma, double* X, double* Y) {
  const int r = m < n ? m : n;
  if (prec == 1) {
    std::vector<Cx<f128_t>> t((size_t)m * n), x, y;
    for (size_t e = 0; e < t.size(); ++e) t[e] = Cx<f128_t>((f128_t)T[2 * e], (f128_t)T[2 * e + 1]);
    std::vector<f128_t> s;
    int sw = svd_general<f128_t>(m, n, t, s, x, y);
    for (int j = 0; j < r; ++j) sigma[j] = (double)s[j];
    for (size_t e = 0; e < (size_t)m * r; ++e) { X[2 * e] = (double)x[e].re; X[2 * e + 1] = (double)x[e].im; }
    for (size_t e = 0; e < (size_t)n * r; ++e) { Y[2 * e] = (double)y[e].re; Y[2 * e + 1] = (double)y[e].im; }
    return sw;
  }
  std::vector<Cx<double>> t((size_t)m * n), x, y;
  for (size_t e = 0; e < t.size(); ++e) t[e] = Cx<double>(T[2 * e], T[2 * e + 1]);
  std::vector<double> s;
  int sw = svd_general<double>(m, n, t, s, x, y);
  for (int j = 0; j < r; ++j) sigma[j] = s[j];
  for (size_t e = 0; e < (size_t)m * r; ++e) { X[2 * e] = x[e].re; X[2 * e + 1] = x[e].im; }
  for (size_t e = 0; e < (size_t)n * r; ++e) { Y[2 * e] = y[e].re; Y[2 * e + 1] = y[e].im; }
  return sw;
}

}  // extern "C"
