// Representable copies of the fused block unitaries (Sec. II's fused
// operators), chosen as close to unitary as their number format allows.
//
// Rounding each entry of a unitary U independently to a finite set of values
// (FP32 for the CUDA-core pass, the three bf16 digits of the tensor-core
// pass) leaves a defect D = Ur^H Ur - I with entries of the order of the
// format's spacing.  The same Ur is applied every period, so the state's
// norm changes by <psi|D|psi> every period, with a sign that repeats: the
// change adds up linearly in the number of periods.  Nearest rounding of
// the bf16 digits gave -1.2e-7 per period at L = 26 (the trace of D summed
// over the 14 passes), which is the whole norm loss measured for that form.
//
// Each real entry x has two representable values bracketing it.  Starting
// from the nearest, a coordinate descent switches single entries to their
// other value whenever that lowers
//     f(Ur) = ||D||_F^2 + tr(D)^2 .
// The trace term is the mean norm change on a maximally mixed window (the
// long-time state); the Frobenius term bounds it for every state.  The
// change of f under one move is known in closed form from (Ur D)_{jk},
// D_kk, tr D and the row norms, and every quantity it needs is updated in
// O(dim) per accepted move by keeping Q = Ur Ur^H beside D.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "sv_block.h"

namespace fsv {

namespace {

// Round to the nearest value with 8 significant bits (bf16 precision, no
// exponent limit: callers keep |x| far inside bf16's range), ties to even.
double bf16_rn(double x) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e;
  const double m = std::frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  return std::ldexp(std::nearbyint(m * 256.0) / 256.0, e);
}

// The 8-significant-bit value next to v (a bf16_rn result) on x's side.
double bf16_other(double x, double v) {
  if (x == v || v == 0.0) return v;
  int e;
  const double m = std::fabs(std::frexp(v, &e));
  const bool up = std::fabs(x) > std::fabs(v);
  // spacing above |v| is 2^(e-8); below a power of two it halves
  const double step = (!up && m == 0.5) ? std::ldexp(1.0, e - 9) : std::ldexp(1.0, e - 8);
  return x > v ? v + step : v - step;
}

// Coordinate descent over the two-valued choice of each real entry.
// A: n x n row-major current values; other[2 (j n + k) + part]: the
// alternative value of the real (part 0) or imaginary (part 1) part of
// A[j][k].  On return A holds the chosen values and other the rejected ones.
// Complex arithmetic is written out on (re, im) pairs: std::complex's
// checked multiplication made this loop several times slower.
void unitary_descent(int n, cd* A, double* other, int max_sweeps) {
  const size_t nn = (size_t)n * n;
  // ar/ai: A; dr/di: D = A^H A - I; qr/qi: Q = A A^H
  std::vector<double> ar(nn), ai(nn), dr(nn), di(nn), qr(nn), qi(nn), mr(n), mi(n), rho(n);
  for (size_t e = 0; e < nn; ++e) {
    ar[e] = A[e].real();
    ai[e] = A[e].imag();
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      double sr = 0, si = 0, tr = 0, ti = 0;
      for (int i = 0; i < n; ++i) {
        const size_t ik = (size_t)i * n + k, il = (size_t)i * n + l;
        sr += ar[ik] * ar[il] + ai[ik] * ai[il];  // conj(A_ik) A_il
        si += ar[ik] * ai[il] - ai[ik] * ar[il];
        const size_t ki = (size_t)k * n + i, li = (size_t)l * n + i;
        tr += ar[ki] * ar[li] + ai[ki] * ai[li];  // A_ki conj(A_li)
        ti += ai[ki] * ar[li] - ar[ki] * ai[li];
      }
      dr[(size_t)k * n + l] = sr - (k == l ? 1.0 : 0.0);
      di[(size_t)k * n + l] = si;
      qr[(size_t)k * n + l] = tr;
      qi[(size_t)k * n + l] = ti;
    }
  double t = 0.0;
  for (int k = 0; k < n; ++k) {
    t += dr[(size_t)k * n + k];
    rho[k] = qr[(size_t)k * n + k];
  }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int moved = 0;
    for (int k = 0; k < n; ++k) {
      // column k of A D
      for (int j = 0; j < n; ++j) {
        double sr = 0, si = 0;
        for (int l = 0; l < n; ++l) {
          const size_t jl = (size_t)j * n + l, lk = (size_t)l * n + k;
          sr += ar[jl] * dr[lk] - ai[jl] * di[lk];
          si += ar[jl] * di[lk] + ai[jl] * dr[lk];
        }
        mr[j] = sr;
        mi[j] = si;
      }
      for (int j = 0; j < n; ++j)
        for (int part = 0; part < 2; ++part) {
          const size_t jk = (size_t)j * n + k;
          const double cur = part == 0 ? ar[jk] : ai[jk];
          double& alt = other[2 * jk + part];
          if (alt == cur) continue;
          // the move a: real (part 0) or imaginary (part 1)
          const double xr = part == 0 ? alt - cur : 0.0, xi = part == 0 ? 0.0 : alt - cur;
          const double a2 = xr * xr + xi * xi;
          const double mre = ar[jk], mim = ai[jk];
          // Re(conj(a) m), Re(conj(a) (A D)_jk)
          const double am = xr * mre + xi * mim;
          const double amd = xr * mr[j] + xi * mi[j];
          const double delta = 2.0 * am + a2;  // change of D_kk (and of tr D, rho_j)
          const double dkk = dr[(size_t)k * n + k];
          const double df = 4.0 * amd + 2.0 * a2 * dkk + 2.0 * a2 * (rho[j] - (mre * mre + mim * mim)) +
                            2.0 * delta * delta + 2.0 * t * delta;
          if (!(df < 0.0)) continue;
          // column k of A D after the move, from the old A and Q and the new
          // D_kk: += (conj(a) m + |a|^2) A[:,k] + a Q[:,j], and a D'_kk at j
          const double cr = xr * mre + xi * mim + a2, ci = xr * mim - xi * mre;
          for (int i = 0; i < n; ++i) {
            const size_t ik = (size_t)i * n + k, ij = (size_t)i * n + j;
            mr[i] += cr * ar[ik] - ci * ai[ik] + xr * qr[ij] - xi * qi[ij];
            mi[i] += cr * ai[ik] + ci * ar[ik] + xr * qi[ij] + xi * qr[ij];
          }
          mr[j] += xr * (dkk + delta);
          mi[j] += xi * (dkk + delta);
          // D row / column k: D_kl += conj(a) A_jl; Q row / column j:
          // Q_ji += a conj(A_ik) (old A)
          for (int l = 0; l < n; ++l) {
            if (l == k) continue;
            const size_t kl = (size_t)k * n + l, lk = (size_t)l * n + k, jl = (size_t)j * n + l;
            dr[kl] += xr * ar[jl] + xi * ai[jl];
            di[kl] += xr * ai[jl] - xi * ar[jl];
            dr[lk] = dr[kl];
            di[lk] = -di[kl];
          }
          dr[(size_t)k * n + k] += delta;
          for (int i = 0; i < n; ++i) {
            if (i == j) continue;
            const size_t ji = (size_t)j * n + i, ij = (size_t)i * n + j, ik = (size_t)i * n + k;
            qr[ji] += xr * ar[ik] + xi * ai[ik];
            qi[ji] += xi * ar[ik] - xr * ai[ik];
            qr[ij] = qr[ji];
            qi[ij] = -qi[ji];
          }
          qr[(size_t)j * n + j] += delta;
          rho[j] += delta;
          t += delta;
          if (part == 0) ar[jk] = alt;
          else ai[jk] = alt;
          alt = cur;
          ++moved;
        }
    }
    if (moved == 0) break;
  }
  for (size_t e = 0; e < nn; ++e) A[e] = cd(ar[e], ai[e]);
}

constexpr int kSweeps = 4;

}  // namespace

void round_unitary_fp32(int dim, const cd* U, float2* out, float4* lead) {
  const size_t nn = (size_t)dim * dim;
  std::vector<cd> A(nn);
  std::vector<double> other(2 * nn);
  std::vector<int> kmax(dim, 0);
  for (int j = 0; j < dim; ++j)
    for (int k = 1; k < dim; ++k)
      if (std::norm(U[(size_t)j * dim + k]) > std::norm(U[(size_t)j * dim + kmax[j]])) kmax[j] = k;
  for (size_t e = 0; e < nn; ++e) {
    const double x[2] = {U[e].real(), U[e].imag()};
    double v[2];
    for (int p = 0; p < 2; ++p) {
      const float f = (float)x[p];
      v[p] = f;
      other[2 * e + p] =
          (double)f == x[p] ? v[p] : (double)std::nextafter(f, x[p] > f ? INFINITY : -INFINITY);
    }
    A[e] = cd(v[0], v[1]);
  }
  if (lead)  // each row's largest entry is applied with its residual: exact
    for (int j = 0; j < dim; ++j) {
      const size_t e = (size_t)j * dim + kmax[j];
      A[e] = U[e];
      other[2 * e] = U[e].real();
      other[2 * e + 1] = U[e].imag();
    }
  unitary_descent(dim, A.data(), other.data(), kSweeps);
  for (size_t e = 0; e < nn; ++e) out[e] = make_float2((float)A[e].real(), (float)A[e].imag());
  if (lead)
    for (int j = 0; j < dim; ++j) {
      const size_t e = (size_t)j * dim + kmax[j];
      const float2 h = make_float2((float)U[e].real(), (float)U[e].imag());
      out[e] = h;
      lead[j] = make_float4((float)(U[e].real() - h.x), (float)(U[e].imag() - h.y), (float)kmax[j],
                            0.f);
    }
}

void round_unitary_digits(int dim, const cd* U, double* digits) {
  const size_t nn = (size_t)dim * dim;
  std::vector<cd> A(nn);
  std::vector<double> other(2 * nn), d2alt(2 * nn);
  for (size_t e = 0; e < nn; ++e) {
    const double x[2] = {U[e].real(), U[e].imag()};
    double v[2];
    for (int p = 0; p < 2; ++p) {
      // u = 2^-7 (u0 + u1 / 256 + u2 / 65536): u0 an integer (the exact
      // level-0 products need it), u1 and u2 with 8 significant bits each
      const double y = x[p] * 128.0;
      const double u0 = std::nearbyint(y);
      const double y1 = (y - u0) * 256.0;
      const double u1 = bf16_rn(y1);
      const double y2 = (y1 - u1) * 256.0;
      double u2 = bf16_rn(y2), o2 = bf16_other(y2, u2);
      if (std::fabs(u2) < 0x1p-90) u2 = o2 = 0.0;  // keep u2 / 2^23 a normal float
      double* d = digits + 3 * (2 * e + p);
      d[0] = u0;
      d[1] = u1;
      d[2] = u2;
      d2alt[2 * e + p] = o2;
      v[p] = (u0 + u1 / 256.0 + u2 / 65536.0) / 128.0;
      other[2 * e + p] = (u0 + u1 / 256.0 + o2 / 65536.0) / 128.0;
    }
    A[e] = cd(v[0], v[1]);
  }
  std::vector<cd> A0 = A;
  unitary_descent(dim, A.data(), other.data(), kSweeps);
  for (size_t e = 0; e < nn; ++e)
    for (int p = 0; p < 2; ++p) {
      const double before = p == 0 ? A0[e].real() : A0[e].imag();
      const double after = p == 0 ? A[e].real() : A[e].imag();
      if (after != before) digits[3 * (2 * e + p) + 2] = d2alt[2 * e + p];
    }
}

void round_passes_parallel(int count, const std::function<void(int)>& job) {
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const int nt = std::min<int>(count, (int)hw);
  if (nt <= 1) {
    for (int k = 0; k < count; ++k) job(k);
    return;
  }
  std::vector<std::thread> th;
  for (int w = 0; w < nt; ++w)
    th.emplace_back([&, w]() {
      for (int k = w; k < count; k += nt) job(k);
    });
  for (auto& x : th) x.join();
}

}  // namespace fsv
