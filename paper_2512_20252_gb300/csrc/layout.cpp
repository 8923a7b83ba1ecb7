// layout.cpp -- the orthant layout of the velocities for the FP32 TMA sweeps.
//
// The sweeps of the mixed path take chunks of KC velocities whose components
// have one sign each (quadrants in 2D, octants in 3D), so that the upwind
// direction along every axis is the same for a whole chunk: the velocities are
// stored grouped by the signs of their components (a zero component counts as
// positive: its flux vanishes either way), in natural order inside a group,
// each group padded to a whole number of chunks.  Padding positions carry
// zero weight and a flux coefficient so large that their equilibrium is
// exactly zero, so their f stays zero.  A layout choice of this library; the
// paper prescribes none.
#include <cmath>
#include <vector>

#include "ctx.h"

namespace ibdvm {

namespace {
constexpr double kPadSpeed = 1e8; // |xi_a| of a padding position: its equilibrium vanishes
}

int orthant_layout(const Geom &G, std::vector<int> &kst, int &nvp) {
  const int D = G.dim;
  std::vector<int> grp[8];
  for (int i = 0; i < G.nv; ++i) {
    int o = 0;
    for (int a = 0; a < D; ++a)
      if (G.xi[3 * i + a] < 0.0) o |= 1 << a;
    grp[o].push_back(i);
  }
  auto padded = [&](int kc) {
    long long n = 0;
    for (const auto &v : grp) n += (static_cast<long long>(v.size()) + kc - 1) / kc * kc;
    return n;
  };
  // The chunk of least sweep time: padded velocities x the sweep's time per
  // padded velocity at that chunk width, relative to the widest (measured on
  // GB300: a lane's per-row work is shared by fewer velocities in narrower
  // chunks).  2D: 192, 128, 64 velocities at 1.00, 1.12, 1.53; 3D: 256, 128
  // at 1.00, 1.32.  The wider chunk on a tie.
  static const int kc2[3] = {192, 128, 64}, w2[3] = {100, 112, 153};
  static const int kc3[2] = {256, 128}, w3[2] = {100, 132};
  const int nc = (D == 3) ? 2 : 3;
  const int *kcs = (D == 3) ? kc3 : kc2, *ws = (D == 3) ? w3 : w2;
  int kc = kcs[0];
  long long best = padded(kcs[0]) * ws[0];
  for (int i = 1; i < nc; ++i) {
    const long long c = padded(kcs[i]) * ws[i];
    if (c < best) {
      best = c;
      kc = kcs[i];
    }
  }
  kst.assign(G.nv, 0);
  int pos = 0;
  for (const auto &v : grp) {
    if (v.empty()) continue;
    for (size_t j = 0; j < v.size(); ++j) kst[v[j]] = pos + static_cast<int>(j);
    pos += (static_cast<int>(v.size()) + kc - 1) / kc * kc;
  }
  nvp = pos;
  return kc;
}

void orthant_tables(const Geom &G, const std::vector<int> &kst, int nvp, int kc, std::vector<float> &vconst,
                    std::vector<uint8_t> &sign) {
  const int D = G.dim;
  vconst.assign(static_cast<size_t>(nvp) * 4, 0.f);
  for (int k = 0; k < nvp; ++k)
    for (int a = 0; a < D; ++a) vconst[4 * static_cast<size_t>(k) + a] = (float)(kPadSpeed * G.dt / G.dx[a]);
  sign.assign(nvp / kc, 0);
  for (int i = 0; i < G.nv; ++i) {
    const size_t k = static_cast<size_t>(kst[i]);
    int o = 0;
    for (int a = 0; a < D; ++a) {
      const double xa = G.xi[3 * i + a];
      vconst[4 * k + a] = (float)(G.dt * std::fabs(xa) / G.dx[a]);
      if (xa < 0.0) o |= 1 << a;
    }
    vconst[4 * k + 3] = (float)G.w[i];
    sign[k / kc] = static_cast<uint8_t>(o);
  }
  if (D == 2) // 2D: (|a_x|, |a_y|, w, 0) per velocity
    for (size_t k = 0; k < static_cast<size_t>(nvp); ++k) {
      vconst[4 * k + 2] = vconst[4 * k + 3];
      vconst[4 * k + 3] = 0.f;
    }
}

} // namespace ibdvm
