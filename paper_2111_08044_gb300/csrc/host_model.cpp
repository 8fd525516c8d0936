// Host-side FP64 construction of the Floquet period: bond Hamiltonians,
// gates exp(-i tau h_b) (Eq. 5 of arXiv 2111.08044), the kick, and kick
// folding.  Independent of the test oracle: gates come from a Jacobi
// eigendecomposition here, from a Taylor series there.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sv_internal.h"

namespace fsv {

namespace {

const cd kI(0.0, 1.0);

// Cyclic Jacobi diagonalisation of a real symmetric n x n matrix a
// (destroyed); q receives the eigenvectors as columns, w the eigenvalues.
void jacobi_sym(int n, double *a, double *q, double *w) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) q[i * n + j] = (i == j);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int r = p + 1; r < n; ++r) {
        double apr = a[p * n + r];
        if (std::fabs(apr) < 1e-300) continue;
        double theta = (a[r * n + r] - a[p * n + p]) / (2.0 * apr);
        double t = (theta >= 0 ? 1.0 : -1.0) /
                   (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // rotate columns p, r
          double akp = a[k * n + p], akr = a[k * n + r];
          a[k * n + p] = c * akp - s * akr;
          a[k * n + r] = s * akp + c * akr;
        }
        for (int k = 0; k < n; ++k) {  // rotate rows p, r
          double apk = a[p * n + k], ark = a[r * n + k];
          a[p * n + k] = c * apk - s * ark;
          a[r * n + k] = s * apk + c * ark;
        }
        for (int k = 0; k < n; ++k) {
          double qkp = q[k * n + p], qkr = q[k * n + r];
          q[k * n + p] = c * qkp - s * qkr;
          q[k * n + r] = s * qkp + c * qkr;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

// Real 8x8 embedding [[A, -B], [B, A]] of the Hermitian 4x4 h = A + iB.
void embed(const cd h[16], double e[64]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double a = h[4 * r + c].real(), b = h[4 * r + c].imag();
      e[8 * r + c] = a;
      e[8 * r + c + 4] = -b;
      e[8 * (r + 4) + c] = b;
      e[8 * (r + 4) + c + 4] = a;
    }
}

// Complex 4x4 from the real embedding's left block column.
void unembed(const double e[64], cd m[16]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) m[4 * r + c] = cd(e[8 * r + c], e[8 * (r + 4) + c]);
}

// Q diag(f) Q^T
void spectral(const double q[64], const double f[8], double out[64]) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double s = 0.0;
      for (int k = 0; k < 8; ++k) s += q[i * 8 + k] * f[k] * q[j * 8 + k];
      out[i * 8 + j] = s;
    }
}

void matmul4(const cd *a, const cd *b, cd *c) {
  cd t[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[4 * i + k] * b[4 * k + j];
      t[4 * i + j] = s;
    }
  std::memcpy(c, t, sizeof(t));
}

// kron(A, B) for 2x2 A (site i, the high bit of r) and B (site i+1).
void kron2(const cd a[4], const cd b[4], cd out[16]) {
  for (int a1 = 0; a1 < 2; ++a1)
    for (int b1 = 0; b1 < 2; ++b1)
      for (int a2 = 0; a2 < 2; ++a2)
        for (int b2 = 0; b2 < 2; ++b2)
          out[4 * (2 * a1 + b1) + (2 * a2 + b2)] = a[2 * a1 + a2] * b[2 * b1 + b2];
}

double field_share(int L, int b, int side, double ew) {
  // share of the on-site fields bond b gives to its left (side 0) or right
  // (side 1) site: h/2, or ew*h at an open end
  int site = b + side;
  bool end = (site == 0) || (site == L - 1);
  return end ? ew : 0.5;
}

}  // namespace

void bond_hamiltonian(int L, int b, double J, double hx, double hz, double ew,
                      cd h[16]) {
  const cd Z[4] = {1, 0, 0, -1}, X[4] = {0, 1, 1, 0}, I2[4] = {1, 0, 0, 1};
  cd t[16];
  double wl = field_share(L, b, 0, ew), wr = field_share(L, b, 1, ew);
  for (int k = 0; k < 16; ++k) h[k] = 0.0;
  kron2(Z, Z, t);
  for (int k = 0; k < 16; ++k) h[k] += J * t[k];
  kron2(X, I2, t);
  for (int k = 0; k < 16; ++k) h[k] += hx * wl * t[k];
  kron2(I2, X, t);
  for (int k = 0; k < 16; ++k) h[k] += hx * wr * t[k];
  kron2(Z, I2, t);
  for (int k = 0; k < 16; ++k) h[k] += hz * wl * t[k];
  kron2(I2, Z, t);
  for (int k = 0; k < 16; ++k) h[k] += hz * wr * t[k];
}

void expm_herm4(const cd h[16], double tau, cd g[16]) {
  double e[64], q[64], w[8], fc[8], fs[8], mc[64], ms[64];
  embed(h, e);
  jacobi_sym(8, e, q, w);
  for (int k = 0; k < 8; ++k) {
    fc[k] = std::cos(tau * w[k]);
    fs[k] = std::sin(tau * w[k]);
  }
  spectral(q, fc, mc);
  spectral(q, fs, ms);
  cd c[16], s[16];
  unembed(mc, c);
  unembed(ms, s);
  for (int k = 0; k < 16; ++k) g[k] = c[k] - kI * s[k];
}

void expm_herm4_frechet(const cd h[16], const cd dh[16], double tau, cd g[16],
                        cd d[16]) {
  // exp(-i tau h) = cos(tau h) - i sin(tau h); both are real functions of h,
  // so their derivatives follow from Daleckii-Krein on the real embedding:
  // Df(H)[E] = Q (F1 o (Q^T E Q)) Q^T with F1_jk = divided difference of f.
  double e[64], q[64], w[8], de[64];
  embed(h, e);
  embed(dh, de);
  jacobi_sym(8, e, q, w);
  double et[64];  // Q^T E Q
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double s = 0.0;
      for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) s += q[a * 8 + i] * de[a * 8 + b] * q[b * 8 + j];
      et[i * 8 + j] = s;
    }
  double outc[64], outs[64];
  for (int pass = 0; pass < 2; ++pass) {
    double m[64];
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) {
        // divided difference of cos / sin written through sum-to-product
        // identities, stable for close and equal eigenvalues
        double mid = 0.5 * tau * (w[i] + w[j]), half = 0.5 * tau * (w[i] - w[j]);
        double sinc = std::fabs(half) < 1e-8 ? 1.0 - half * half / 6.0 : std::sin(half) / half;
        double f1 = pass == 0 ? -tau * std::sin(mid) * sinc : tau * std::cos(mid) * sinc;
        m[i * 8 + j] = f1 * et[i * 8 + j];
      }
    double *out = pass == 0 ? outc : outs;
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) {
        double s = 0.0;
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b) s += q[i * 8 + a] * m[a * 8 + b] * q[j * 8 + b];
        out[i * 8 + j] = s;
      }
  }
  cd c[16], s[16];
  unembed(outc, c);
  unembed(outs, s);
  for (int k = 0; k < 16; ++k) d[k] = c[k] - kI * s[k];
  expm_herm4(h, tau, g);
}

void kick_matrix(double theta, cd r[4]) {
  // exp(-i theta X) = cos(theta) I - i sin(theta) X, since X^2 = I
  double c = std::cos(theta), s = std::sin(theta);
  r[0] = c;
  r[1] = cd(0.0, -s);
  r[2] = cd(0.0, -s);
  r[3] = c;
}

bool params_valid(int L, const sv_floquet_params &p, std::string *why) {
  auto bad = [&](const char *m) {
    if (why) *why = m;
    return false;
  };
  if (L < 2 || L > 34) return bad("L must be in 2..34");
  if (p.K < 1 || p.K > 1024) return bad("K must be in 1..1024");
  if (p.first_layer != 0 && p.first_layer != 1) return bad("first_layer must be 0 or 1");
  if (!std::isfinite(p.J) || !std::isfinite(p.hx) || !std::isfinite(p.hz) ||
      !std::isfinite(p.T) || !std::isfinite(p.theta) ||
      !std::isfinite(p.edge_field_weight))
    return bad("non-finite parameter");
  if (p.mode != SV_MODE_PLAIN && p.mode != SV_MODE_BLOCK && p.mode != SV_MODE_MULTIGATE)
    return bad("unknown mode");
  if (p.renorm_every < 0) return bad("renorm_every must be >= 0");
  if (p.n_period_params < 0) return bad("n_period_params must be >= 0");
  if (p.n_period_params > 0 && !p.theta_p && !p.hx_p)
    return bad("n_period_params > 0 needs theta_p or hx_p");
  if (p.inverse != 0 && p.inverse != 1) return bad("inverse must be 0 or 1");
  if (p.h_bonds) {
    if (p.n_period_params > 0) return bad("h_bonds needs n_period_params = 0");
    if (p.renorm_every > 0) return bad("h_bonds needs renorm_every = 0");
    for (int b = 0; b < L - 1; ++b) {
      const double *m = p.h_bonds + 32 * (size_t)b;
      double scale = 0.0;
      for (int k = 0; k < 32; ++k) {
        if (!std::isfinite(m[k])) return bad("non-finite h_bonds entry");
        scale = std::max(scale, std::fabs(m[k]));
      }
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          const double dre = m[2 * (4 * r + c)] - m[2 * (4 * c + r)];
          const double dim = m[2 * (4 * r + c) + 1] + m[2 * (4 * c + r) + 1];
          if (std::fabs(dre) > 1e-12 * (1.0 + scale) || std::fabs(dim) > 1e-12 * (1.0 + scale))
            return bad("h_bonds entry is not Hermitian");
        }
    }
  }
  if (p.inverse && p.n_period_params > 0)
    return bad("inverse periods need fixed parameters (n_period_params = 0)");
  return true;
}

std::vector<Gate2> period_gates(int L, const sv_floquet_params &p, double theta,
                                double hx) {
  const double tau = p.T / p.K;
  std::vector<cd> gb((size_t)16 * (L - 1));
  for (int b = 0; b < L - 1; ++b) {
    cd h[16];
    if (p.h_bonds) {
      for (int k = 0; k < 16; ++k) h[k] = cd(p.h_bonds[32 * b + 2 * k], p.h_bonds[32 * b + 2 * k + 1]);
    } else {
      bond_hamiltonian(L, b, p.J, hx, p.hz, p.edge_field_weight, h);
    }
    expm_herm4(h, tau, &gb[16 * (size_t)b]);
  }
  std::vector<Gate2> out;
  for (int s = 0; s < p.K; ++s)
    for (int layer = 0; layer < 2; ++layer) {
      int parity = layer == 0 ? p.first_layer : 1 - p.first_layer;
      for (int b = parity; b < L - 1; b += 2) {
        Gate2 g;
        g.bond = b;
        std::memcpy(g.m, &gb[16 * (size_t)b], sizeof(g.m));
        out.push_back(g);
      }
    }
  // a2: the kick on site i commutes with every later gate of the period
  // (none touches i), so it folds into the last gate on i.
  cd R[4], I2[4] = {1, 0, 0, 1}, F[16];
  kick_matrix(theta, R);
  std::vector<int> last(L, -1);
  for (int g = 0; g < (int)out.size(); ++g) {
    last[out[g].bond] = g;
    last[out[g].bond + 1] = g;
  }
  for (int i = 0; i < L; ++i) {
    Gate2 &g = out[last[i]];
    if (g.bond == i) {
      kron2(R, I2, F);
      g.epi |= EPI_X_HI;
    } else {
      kron2(I2, R, F);
      g.epi |= EPI_X_LO;
    }
    matmul4(F, g.m, g.m);
  }
  out.back().epi |= EPI_DIAG;
  if (p.inverse) {
    // U_F^dagger (the echo of Sec. V): the same gates in reverse order, each
    // replaced by its adjoint (the folded kicks are then undone first).  Each
    // site's <X> is read at its last gate of the new order, the diagonal part
    // at the last gate, so every measurement sees the period's final state.
    std::reverse(out.begin(), out.end());
    for (Gate2 &g : out) {
      cd t[16];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) t[4 * r + c] = std::conj(g.m[4 * c + r]);
      std::memcpy(g.m, t, sizeof(t));
      g.epi = 0;
    }
    std::vector<int> last2(L, -1);
    for (int g = 0; g < (int)out.size(); ++g) {
      last2[out[g].bond] = g;
      last2[out[g].bond + 1] = g;
    }
    for (int i = 0; i < L; ++i) out[last2[i]].epi |= out[last2[i]].bond == i ? EPI_X_HI : EPI_X_LO;
    out.back().epi |= EPI_DIAG;
  }
  // a general two-site chain has no fused per-period measurement
  if (p.h_bonds)
    for (Gate2 &g : out) g.epi = 0;
  return out;
}

std::vector<AdjOp> adjoint_period_ops(int L, const sv_floquet_params &p, double theta,
                                      double hx) {
  auto dagger4 = [](const cd *m, cd *out) {
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) out[4 * r + c] = std::conj(m[4 * c + r]);
  };
  std::vector<AdjOp> ops;
  // kick: exp(-i theta X) on each site; d/dtheta R R^dagger = -i X
  cd R[4], I2[4] = {1, 0, 0, 1}, X[4] = {0, 1, 1, 0}, mX[4], O[16], t1[16], t2[16];
  kick_matrix(theta, R);
  for (int k = 0; k < 4; ++k) mX[k] = -kI * X[k];
  for (int i = 0; i + 1 < L; i += 2) {
    AdjOp op;
    op.bond = i;
    op.kind = 0;
    kron2(R, R, O);
    dagger4(O, op.odag);
    kron2(mX, I2, t1);
    kron2(I2, mX, t2);
    for (int k = 0; k < 16; ++k) op.d[k] = t1[k] + t2[k];
    ops.push_back(op);
  }
  if (L % 2 == 1) {
    AdjOp op;
    op.bond = L - 2;
    op.kind = 0;
    kron2(I2, R, O);
    dagger4(O, op.odag);
    kron2(I2, mX, op.d);
    ops.push_back(op);
  }
  // gates: G_b = exp(-i tau h_b(hx)), dh_b/dhx is h_b at J = hz = 0, hx = 1
  const double tau = p.T / p.K;
  std::vector<AdjOp> gate_ops(L - 1);
  for (int b = 0; b < L - 1; ++b) {
    cd h[16], dh[16], g[16], dg[16], gd[16];
    bond_hamiltonian(L, b, p.J, hx, p.hz, p.edge_field_weight, h);
    bond_hamiltonian(L, b, 0.0, 1.0, 0.0, p.edge_field_weight, dh);
    expm_herm4_frechet(h, dh, tau, g, dg);
    AdjOp &op = gate_ops[b];
    op.bond = b;
    op.kind = 1;
    dagger4(g, gd);
    std::memcpy(op.odag, gd, sizeof(gd));
    matmul4(dg, gd, op.d);
  }
  for (int s = p.K - 1; s >= 0; --s)
    for (int layer = 1; layer >= 0; --layer) {
      const int parity = layer == 0 ? p.first_layer : 1 - p.first_layer;
      for (int b = parity; b < L - 1; b += 2) ops.push_back(gate_ops[b]);
    }
  return ops;
}

double site_field_share(int L, int i, double ew) {
  // the bonds (i-1, i) and (i, i+1) each give site i its share of the fields
  double w = 0.0;
  if (i >= 1) w += field_share(L, i - 1, 1, ew);
  if (i + 1 <= L - 1) w += field_share(L, i, 0, ew);
  return w;
}

Observable observable(int L, const sv_floquet_params &p) {
  Observable o;
  o.L = L;
  if (p.h_bonds) {
    o.general = true;
    o.h.resize(16 * (size_t)(L - 1));
    for (size_t k = 0; k < o.h.size(); ++k) o.h[k] = cd(p.h_bonds[2 * k], p.h_bonds[2 * k + 1]);
    return o;
  }
  o.J = p.J;
  o.cx.assign(L, 0.0);
  o.cz.assign(L, 0.0);
  for (int i = 0; i < L; ++i) {
    const double w = site_field_share(L, i, p.edge_field_weight);
    o.cx[i] = p.hx * w;
    o.cz[i] = p.hz * w;
  }
  return o;
}

}  // namespace fsv
