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
  int kc;
  if (D == 3) {
    // 256-velocity chunks unless 128 wastes clearly less padding
    kc = (padded(256) <= padded(128) + padded(128) / 32) ? 256 : 128;
  } else {
    // the chunk of least padding among 192, 128 and 64 (the larger on a tie)
    kc = 192;
    for (int c : {128, 64})
      if (padded(c) < padded(kc)) kc = c;
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
