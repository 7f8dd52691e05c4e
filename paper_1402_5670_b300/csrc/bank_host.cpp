// Host FP64 construction of the digital shearlet filter bank.
//
// Each filter is evaluated directly from the closed form of its frequency response,
// i.e. the DTFT of the paper's spatial construction sampled on the N-grid (the DFT of
// the periodically folded filter). The spatial operators have these responses:
//
//   h_j, g_j (eq. lowhigh, Sec. 3.1):   h_hat_j(w) = prod_{i<j} H(2^i w),
//                                       g_hat_j(w) = G(2^{j-1} w) h_hat_{j-1}(w),
//                                       G(w) = H(w + pi)       (g(n) = (-1)^n h(n), Sec. 5.1)
//   p_j (eq. ext_noshear_alpha):        P(2^{J-j-1} w1, 2^{J-j+d} w2)
//   W_j = g_{J-j} (x) h_{J-j+d}:        g_hat_{J-j}(w1) h_hat_{J-j+d}(w2)
//   digital shear S^d_{k/2^d} (eqs. dshear1_alpha, dshear2_alpha): upsampling x1 by
//     2^d, filtering with 2^d h_d, resampling by S_k, filtering with h_d and keeping
//     every 2^d-th sample multiply-and-alias the response:
//       (S f)^(w1, w2) = sum_{r=0}^{2^d-1} h_hat_d(o_r)^2 f_hat(w1, w2 - k o_r),
//       o_r = (w1 + 2 pi r) / 2^d.
//   2D filter (Def. digitSH_alpha):     psi_hat_{j,k}(w) = g_hat_{J-j}(w1) Phi_{j,k}(w1, w2)
//   3D filter (Def. 3DdigitSH_alpha):   g_hat_{J-j}(w1) Phi_{j,k1}(w1, w2) Phi_{j,k2}(w1, w3)
//   with Phi_{j,k}(a, b) = sum_r h_hat_d(o_r)^2 h_hat_{J-j+d}(b - k o_r)
//                                P(2^{J-j-1} a, 2^{J-j+d} (b - k o_r)).
//   Second cone / pyramids: axis permutations (Sec. 3.4 eq. convolution01; Sec. 3.3.1).
//
// The design constants of H (maximally flat, half power at half band, Sec. 5.1) and of
// the fan filter P (maximally flat diamond polynomial, modulated into a fan) are solved
// for from their defining conditions below rather than typed in.

#include "bank_host.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <string>

namespace sl {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// H(w) = 1 + a s^3 + b s^4 with s = sin^2(w/2): H(pi) = 0 and H(pi/2) = 1/sqrt(2).
struct LowpassDesign {
  double a3, a4;
  LowpassDesign() {
    // rows: [s^3 s^4 | rhs] at s = 1 and s = 1/2
    const double m00 = 1.0, m01 = 1.0, r0 = -1.0;
    const double m10 = 0.125, m11 = 0.0625, r1 = 1.0 / std::sqrt(2.0) - 1.0;
    const double det = m00 * m11 - m01 * m10;
    a3 = (r0 * m11 - m01 * r1) / det;
    a4 = (m00 * r1 - r0 * m10) / det;
  }
};

// M(t) = 1/2 + sum_i c_{2i+1} t^{2i+1} with M'(t) = C (1 - t^2)^3 and M(1) = 1.
struct FanDesign {
  double c[4];  // c1, c3, c5, c7
  FanDesign() {
    const double binom[4] = {1.0, 3.0, 3.0, 1.0};
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s += binom[i] * ((i & 1) ? -1.0 : 1.0) / (2 * i + 1);
    const double C = 0.5 / s;
    for (int i = 0; i < 4; ++i) c[i] = C * binom[i] * ((i & 1) ? -1.0 : 1.0) / (2 * i + 1);
  }
};

const LowpassDesign& lp() { static const LowpassDesign d; return d; }
const FanDesign& fan() { static const FanDesign d; return d; }

inline double H_of_s(double s) {
  const LowpassDesign& d = lp();
  const double s3 = s * s * s;
  return 1.0 + d.a3 * s3 + d.a4 * s3 * s;
}

inline double pow2(int e) { return std::ldexp(1.0, e); }

}  // namespace

// DTFT of symmetric taps h(-m..m): h(0) + 2 sum_{n>0} h(n) cos(n w) (real).
static double user_lowpass(const std::vector<double>& h, double w) {
  const int m = ((int)h.size() - 1) / 2;
  const double c1 = std::cos(w);
  double acc = h[m], cp = 1.0, cn = c1;  // cos((n-1) w), cos(n w) by recurrence
  for (int n = 1; n <= m; ++n) {
    acc += 2.0 * h[m + n] * cn;
    const double nx = 2.0 * c1 * cn - cp;
    cp = cn;
    cn = nx;
  }
  return acc;
}

// DTFT of point-symmetric 2D taps: sum p(n1, n2) cos(n1 w1 + n2 w2) (real).
static double user_fan(const FilterDesign& D, double w1, double w2) {
  const int m1 = (D.pr - 1) / 2, m2 = (D.pc - 1) / 2;
  double c1[65], s1[65], c2[65], s2[65];  // cos, sin of n w for n = 0..m
  c1[0] = 1.0, s1[0] = 0.0, c2[0] = 1.0, s2[0] = 0.0;
  const double a = std::cos(w1), b = std::sin(w1), c = std::cos(w2), e = std::sin(w2);
  for (int n = 1; n <= m1; ++n) {
    c1[n] = c1[n - 1] * a - s1[n - 1] * b;
    s1[n] = s1[n - 1] * a + c1[n - 1] * b;
  }
  for (int n = 1; n <= m2; ++n) {
    c2[n] = c2[n - 1] * c - s2[n - 1] * e;
    s2[n] = s2[n - 1] * c + c2[n - 1] * e;
  }
  double acc = 0.0;
  for (int i = 0; i < D.pr; ++i) {
    const int n1 = i - m1;
    const double ca = c1[n1 < 0 ? -n1 : n1], sa = n1 < 0 ? -s1[-n1] : s1[n1];
    const double* row = D.p.data() + (size_t)i * D.pc;
    for (int k = 0; k < D.pc; ++k) {
      const int n2 = k - m2;
      const double cb = c2[n2 < 0 ? -n2 : n2], sb = n2 < 0 ? -s2[-n2] : s2[n2];
      acc += row[k] * (ca * cb - sa * sb);
    }
  }
  return acc;
}

double resp_lowpass(const FilterDesign* D, double w) {
  if (D && !D->h.empty()) return user_lowpass(D->h, w);
  return H_of_s(0.5 * (1.0 - std::cos(w)));
}

double resp_lowpass_j(const FilterDesign* D, int j, double w) {
  double p = 1.0;
  for (int i = 0; i < j; ++i) p *= resp_lowpass(D, pow2(i) * w);
  return p;
}

// G(w) = H(w + pi): g(n) = (-1)^n h(n)
static double resp_highpass(const FilterDesign* D, double w) {
  if (D && !D->h.empty()) return user_lowpass(D->h, w + kPi);
  return H_of_s(0.5 * (1.0 + std::cos(w)));
}

double resp_highpass_j(const FilterDesign* D, int j, double w) {
  return resp_highpass(D, pow2(j - 1) * w) * resp_lowpass_j(D, j - 1, w);
}

double resp_fan(const FilterDesign* D, double w1, double w2) {
  if (D && !D->p.empty()) return user_fan(*D, w1, w2);
  const FanDesign& f = fan();
  const double t = 0.5 * (std::cos(w2) - std::cos(w1));
  const double t2 = t * t;
  return 0.5 + t * (f.c[0] + t2 * (f.c[1] + t2 * (f.c[2] + t2 * f.c[3])));
}

std::string check_design(const FilterDesign& d) {
  if (!d.h.empty()) {
    const int n = (int)d.h.size();
    if (n % 2 == 0 || n > 129) return "qmf taps: odd length up to 129 required";
    double mx = 0.0;
    for (double v : d.h) mx = std::max(mx, std::fabs(v));
    if (!(mx > 0.0) || !std::isfinite(mx)) return "qmf taps must be finite and not all zero";
    for (int i = 0; i < n; ++i)
      if (std::fabs(d.h[i] - d.h[n - 1 - i]) > 1e-12 * mx)
        return "qmf taps must be symmetric (h(-n) = h(n)), so that the spectra are real";
  }
  if (!d.p.empty()) {
    if (d.pr % 2 == 0 || d.pc % 2 == 0 || d.pr > 65 || d.pc > 65 ||
        (size_t)d.pr * d.pc != d.p.size())
      return "fan taps: odd sizes up to 65 x 65 required";
    double mx = 0.0;
    for (double v : d.p) mx = std::max(mx, std::fabs(v));
    if (!(mx > 0.0) || !std::isfinite(mx)) return "fan taps must be finite and not all zero";
    for (size_t i = 0; i < d.p.size(); ++i)
      if (std::fabs(d.p[i] - d.p[d.p.size() - 1 - i]) > 1e-12 * mx)
        return "fan taps must be point-symmetric (P(-n) = P(n)), so that the spectra are real";
  }
  return "";
}

// Phi_{j,k}(a, b) for scale j with shear level d, J scales.
static double phi_resp(const FilterDesign* D, int J, int j, int d, int k, double a, double b) {
  const int m = J - j + d;
  const double pa = pow2(J - j - 1) * a;
  const int nr = 1 << d;
  double acc = 0.0;
  for (int r = 0; r < nr; ++r) {
    const double o = (a + 2.0 * kPi * r) / nr;
    const double wd = resp_lowpass_j(D, d, o);
    const double eta = b - k * o;
    acc += wd * wd * resp_lowpass_j(D, m, eta) * resp_fan(D, pa, pow2(m) * eta);
  }
  return acc;
}

std::vector<FilterDesc> enumerate_filters(const BankSpec& s) {
  std::vector<FilterDesc> out;
  out.push_back({-1, 0, 0, 0});
  if (s.kind == kWavelets) {  // per scale, coarse to fine: g (x) h, h (x) g, g (x) g
    for (int j = 0; j < s.J; ++j)
      for (int o = 1; o <= 3; ++o) out.push_back({j, o, 0, 0});
    return out;
  }
  for (int j = 0; j < s.J; ++j) {
    const int e = 1 << s.d[j];
    if (s.ndim == 2) {
      for (int k = -e; k <= e; ++k) out.push_back({j, 1, k, 0});
      for (int k = -e; k <= e; ++k)
        if (s.full || std::abs(k) != e) out.push_back({j, 2, k, 0});
    } else {
      for (int pyr = 1; pyr <= 3; ++pyr)
        for (int k1 = -e; k1 <= e; ++k1)
          for (int k2 = -e; k2 <= e; ++k2) {
            bool keep = true;
            if (!s.full) {
              if (pyr == 2) keep = std::abs(k1) != e;
              if (pyr == 3) keep = std::abs(k1) != e && std::abs(k2) != e;
            }
            if (keep) out.push_back({j, pyr, k1, k2});
          }
    }
  }
  return out;
}

// (principal, k1 axis, k2 axis) of the three pyramids.
static const int kPyr[4][3] = {{0, 0, 0}, {0, 1, 2}, {1, 0, 2}, {2, 0, 1}};

BankEvaluator::BankEvaluator(const BankSpec& s) : spec_(s), filt_(enumerate_filters(s)) {
  for (int j = 0; j < s.J; ++j) kmax_ = std::max(kmax_, 1 << s.d[j]);
  if (s.ndim == 3) build_3d_tables();
}

int BankEvaluator::phi_index(int scale, int k, int pa, int pb) const {
  return ((scale * (2 * kmax_ + 1) + (k + kmax_)) * 3 + pa) * 3 + pb;
}

void BankEvaluator::build_3d_tables() {
  const BankSpec& s = spec_;
  const FilterDesign* D = s.design.get();
  g1_.assign(s.J * 3, {});
  phi2_.assign(s.J * (2 * kmax_ + 1) * 9, {});
  for (int j = 0; j < s.J; ++j) {
    for (int ax = 0; ax < 3; ++ax) {
      std::vector<double>& t = g1_[j * 3 + ax];
      t.resize(s.dims[ax]);
      for (int64_t i = 0; i < s.dims[ax]; ++i)
        t[i] = resp_highpass_j(D, s.J - j, 2.0 * kPi * i / s.dims[ax]);
    }
    const int e = 1 << s.d[j];
    for (int pyr = 1; pyr <= 3; ++pyr) {
      const int p = kPyr[pyr][0];
      for (int which = 1; which <= 2; ++which) {
        const int q = kPyr[pyr][which];
        for (int k = -e; k <= e; ++k) {
          std::vector<double>& t = phi2_[phi_index(j, k, p, q)];
          if (!t.empty()) continue;
          const int64_t np = s.dims[p], nq = s.dims[q];
          t.resize(np * nq);
          for (int64_t ip = 0; ip < np; ++ip)
            for (int64_t iq = 0; iq < nq; ++iq)
              t[ip * nq + iq] = phi_resp(D, s.J, j, s.d[j], k, 2.0 * kPi * ip / np,
                                         2.0 * kPi * iq / nq);
        }
      }
    }
  }
}

void BankEvaluator::eval_2d(const FilterDesc& f, double* out) const {
  const BankSpec& s = spec_;
  const FilterDesign* D = s.design.get();
  const int64_t n0 = s.dims[0], n1 = s.dims[1], nh = s.nh();
  if (f.scale < 0) {
    for (int64_t i0 = 0; i0 < n0; ++i0) {
      const double a = resp_lowpass_j(D, s.J, 2.0 * kPi * i0 / n0);
      for (int64_t i1 = 0; i1 < nh; ++i1)
        out[i0 * nh + i1] = a * resp_lowpass_j(D, s.J, 2.0 * kPi * i1 / n1);
    }
    return;
  }
  if (s.kind == kWavelets) {
    // the a trous stationary wavelet filters at level a = J - j (eq. lowhigh's h_a and
    // g_a on each axis): cone 1 = g_a(xi_1) h_a(xi_2), 2 = h_a(xi_1) g_a(xi_2), 3 = g_a g_a
    const int a = s.J - f.scale;
    std::vector<double> r1(nh);
    for (int64_t i1 = 0; i1 < nh; ++i1) {
      const double x1 = 2.0 * kPi * i1 / n1;
      r1[i1] = f.cone == 1 ? resp_lowpass_j(D, a, x1) : resp_highpass_j(D, a, x1);
    }
    for (int64_t i0 = 0; i0 < n0; ++i0) {
      const double x0 = 2.0 * kPi * i0 / n0;
      const double r0 = f.cone == 2 ? resp_lowpass_j(D, a, x0) : resp_highpass_j(D, a, x0);
      for (int64_t i1 = 0; i1 < nh; ++i1) out[i0 * nh + i1] = r0 * r1[i1];
    }
    return;
  }
  const int j = f.scale, d = s.d[j];
  for (int64_t i0 = 0; i0 < n0; ++i0) {
    const double x0 = 2.0 * kPi * i0 / n0;
    for (int64_t i1 = 0; i1 < nh; ++i1) {
      const double x1 = 2.0 * kPi * i1 / n1;
      const double a = f.cone == 1 ? x0 : x1;  // principal axis
      const double b = f.cone == 1 ? x1 : x0;
      out[i0 * nh + i1] = resp_highpass_j(D, s.J - j, a) * phi_resp(D, s.J, j, d, f.k1, a, b);
    }
  }
}

void BankEvaluator::eval_3d(const FilterDesc& f, double* out) const {
  const BankSpec& s = spec_;
  const FilterDesign* D = s.design.get();
  const int64_t n0 = s.dims[0], n1 = s.dims[1], n2 = s.dims[2], nh = s.nh();
  if (f.scale < 0) {
    std::vector<double> l[3];
    for (int ax = 0; ax < 3; ++ax) {
      l[ax].resize(s.dims[ax]);
      for (int64_t i = 0; i < s.dims[ax]; ++i)
        l[ax][i] = resp_lowpass_j(D, s.J, 2.0 * kPi * i / s.dims[ax]);
    }
    for (int64_t i0 = 0; i0 < n0; ++i0)
      for (int64_t i1 = 0; i1 < n1; ++i1)
        for (int64_t i2 = 0; i2 < nh; ++i2)
          out[(i0 * n1 + i1) * nh + i2] = l[0][i0] * l[1][i1] * l[2][i2];
    return;
  }
  const int p = kPyr[f.cone][0], b = kPyr[f.cone][1], c = kPyr[f.cone][2];
  const std::vector<double>& g = g1_[f.scale * 3 + p];
  const std::vector<double>& t1 = phi2_[phi_index(f.scale, f.k1, p, b)];
  const std::vector<double>& t2 = phi2_[phi_index(f.scale, f.k2, p, c)];
  const int64_t nb = s.dims[b], nc = s.dims[c];
  int64_t idx[3];
  for (idx[0] = 0; idx[0] < n0; ++idx[0])
    for (idx[1] = 0; idx[1] < n1; ++idx[1]) {
      double* row = out + (idx[0] * n1 + idx[1]) * nh;
      for (idx[2] = 0; idx[2] < nh; ++idx[2]) {
        const int64_t ip = idx[p], ib = idx[b], ic = idx[c];
        row[idx[2]] = g[ip] * t1[ip * nb + ib] * t2[ip * nc + ic];
      }
    }
  (void)n2;
}

void BankEvaluator::eval(int j, double* out) const {
  if (spec_.ndim == 2) eval_2d(filt_[j], out);
  else eval_3d(filt_[j], out);
}

// Weight of a half-spectrum column in sums over the full grid.
static inline double half_weight(int64_t i_last, int64_t n_last) {
  return (i_last == 0 || 2 * i_last == n_last) ? 1.0 : 2.0;
}

bool build_host_bank(const BankSpec& s, bool want_psi32, HostBank* out, std::string* err) {
  BankEvaluator ev(s);
  const int R = ev.R();
  const int64_t Nh = s.Nh(), nh = s.nh(), nl = s.n_last();
  out->filt = ev.filters();
  unsigned hw = std::thread::hardware_concurrency();
  int nthreads = (int)std::max(1u, std::min(hw ? hw : 4u, 64u));
  nthreads = std::min(nthreads, R);

  // Pass 1: Psi = sum_j psi_hat_j^2 and the full-grid energies of each filter.
  std::vector<std::vector<double>> psi_part(nthreads);
  std::vector<double> energy(R, 0.0);
  {
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t)
      th.emplace_back([&, t]() {
        std::vector<double>& acc = psi_part[t];
        acc.assign(Nh, 0.0);
        std::vector<double> v(Nh);
        for (int j; (j = next.fetch_add(1)) < R;) {
          ev.eval(j, v.data());
          double e = 0.0;
          for (int64_t i = 0; i < Nh; ++i) {
            const double q = v[i] * v[i];
            acc[i] += q;
            e += half_weight(i % nh, nl) * q;
          }
          energy[j] = e;
        }
      });
    for (auto& x : th) x.join();
  }
  std::vector<double> Psi(Nh, 0.0);
  for (int t = 0; t < nthreads; ++t)
    for (int64_t i = 0; i < Nh; ++i) Psi[i] += psi_part[t][i];
  psi_part.clear();
  double mx = 0.0, mn = 1e300;
  for (int64_t i = 0; i < Nh; ++i) {
    mx = std::max(mx, Psi[i]);
    mn = std::min(mn, Psi[i]);
  }
  if (!(mn > 0.0) || !std::isfinite(mx)) {
    if (err) *err = "frame weight Psi is not positive on the grid";
    return false;
  }
  out->scale = 1.0 / std::sqrt(mx);
  out->A = mn / mx;
  out->B = 1.0;
  out->invPsi.resize(Nh);
  for (int64_t i = 0; i < Nh; ++i) out->invPsi[i] = mx / Psi[i];
  out->norms.resize(R);
  for (int j = 0; j < R; ++j) out->norms[j] = std::sqrt(energy[j] / mx / (double)s.N());

  // Pass 2: the normalised FP32 bank.
  if (want_psi32) {
    out->psi32.assign((size_t)R * Nh, 0.0f);
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t)
      th.emplace_back([&]() {
        std::vector<double> v(Nh);
        for (int j; (j = next.fetch_add(1)) < R;) {
          ev.eval(j, v.data());
          float* dst = out->psi32.data() + (size_t)j * Nh;
          for (int64_t i = 0; i < Nh; ++i) dst[i] = (float)(v[i] * out->scale);
        }
      });
    for (auto& x : th) x.join();
  }
  return true;
}

}  // namespace sl
