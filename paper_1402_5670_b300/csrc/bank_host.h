// Host-side (FP64) construction of the digital shearlet filter bank from the closed
// form of each filter's frequency response. Internal to libshearlet.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

namespace sl {

struct FilterDesc {
  int scale;  // 0..J-1, -1 for the lowpass
  int cone;   // 2D: cone 1/2; 3D: pyramid 1..3; wavelets: 1 = g (x) h, 2 = h (x) g,
              // 3 = g (x) g; 0 for the lowpass
  int k1;     // shear (2D) or first shear (3D)
  int k2;     // second shear (3D), 0 in 2D
};

// User-supplied filters (Sec. 4.1: the QMF lowpass and the 2D fan filter are inputs of
// the construction). Empty vectors select the built-in designs.
struct FilterDesign {
  std::vector<double> h;  // taps h(-m..m), odd length, symmetric
  std::vector<double> p;  // taps P(n1, n2), [pr][pc] row-major, centred, point-symmetric
  int pr = 0, pc = 0;     // (axis 0 of P pairs with xi_1, axis 1 with xi_2)
};

// The filter systems a bank can hold.
enum BankKind {
  kShearlets = 0,  // the digital shearlet system (Defs. digitSH_alpha, 3DdigitSH_alpha)
  kWavelets = 1    // the separable stationary wavelet system on the same QMF (2D only)
};

struct BankSpec {
  std::shared_ptr<const FilterDesign> design;  // null: built-in filters
  int kind = kShearlets;
  int ndim = 2;
  int64_t dims[3] = {1, 1, 1};
  int J = 1;
  int d[8] = {0};
  bool full = false;

  int64_t n_last() const { return dims[ndim - 1]; }
  int64_t nh() const { return dims[ndim - 1] / 2 + 1; }
  int64_t N() const { return dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1); }
  int64_t Nh() const { return N() / n_last() * nh(); }
};

// Enumerate the filters of a system in the library's order.
std::vector<FilterDesc> enumerate_filters(const BankSpec& s);

// Evaluator of unnormalised filter responses on the half-spectrum grid.
class BankEvaluator {
 public:
  explicit BankEvaluator(const BankSpec& s);
  const BankSpec& spec() const { return spec_; }
  const std::vector<FilterDesc>& filters() const { return filt_; }
  int R() const { return (int)filt_.size(); }
  // out[Nh] = unnormalised psi_hat_j on the half spectrum [n0][..][nh].
  void eval(int j, double* out) const;

 private:
  BankSpec spec_;
  std::vector<FilterDesc> filt_;
  // 3D factor tables: g_hat_{J-j} per (scale, axis) and Phi_hat_{j,k} per
  // (scale, shear, principal axis, secondary axis) on the full 2D grid.
  std::vector<std::vector<double>> g1_;   // [scale*3 + axis][n_axis]
  std::vector<std::vector<double>> phi2_; // index via phi_index()
  int phi_index(int scale, int k, int pa, int pb) const;
  int kmax_ = 0;
  void build_3d_tables();
  void eval_2d(const FilterDesc& f, double* out) const;
  void eval_3d(const FilterDesc& f, double* out) const;
};

// Result of a full host build: normalised FP32 half spectra and FP64 frame data.
struct HostBank {
  std::vector<FilterDesc> filt;
  std::vector<float> psi32;     // [R][Nh] normalised
  std::vector<double> invPsi;   // [Nh] 1 / Psi (normalised)
  std::vector<double> norms;    // [R] ||psi_j||_2
  double scale = 1.0;           // 1 / sqrt(max Psi_unnormalised)
  double A = 0.0, B = 0.0;
};

// Evaluate all filters (multithreaded), normalise, and fill HostBank.
// want_psi32 = false skips the FP32 bank (host-only banks).
bool build_host_bank(const BankSpec& s, bool want_psi32, HostBank* out, std::string* err);

// 1D/2D responses of the filters of design D (null: the built-in closed forms).
double resp_lowpass(const FilterDesign* D, double w);             // h_hat(w)
double resp_lowpass_j(const FilterDesign* D, int j, double w);    // h_hat_j(w), eq. lowhigh
double resp_highpass_j(const FilterDesign* D, int j, double w);   // g_hat_j(w), eq. lowhigh
double resp_fan(const FilterDesign* D, double w1, double w2);     // P(w1, w2)

// Checks user taps: odd sizes, symmetric h, point-symmetric P (relative 1e-12), sizes
// h <= 129 and P <= 65 x 65. Returns an empty string or the reason.
std::string check_design(const FilterDesign& d);

}  // namespace sl
