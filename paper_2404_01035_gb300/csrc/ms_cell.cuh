// One explicit grand-potential step for one cell, generic over
//   - the scalar S (float, double, or a forward-mode Dual for the adjoint),
//   - the accessor Acc that supplies the stencil (shared-memory tiles in the
//     forward kernel, global memory with seeded duals in the adjoint).
//
// Steps, in order (MICROSIM paper, arXiv 2404.01035, Sec. 2.1):
//   S1/S2  face values, face gradients and the anisotropic face flux
//          J_a = da/dgrad phi_a = -sum_b phi_b g_ab(q_ab), q_ab = phi_a grad phi_b
//          - phi_b grad phi_a, g = dA/dq (Eqs. Eqn_a, aniso_eqn);
//   S3     divergence of J and the centre term da/dphi_a = sum_b g_ab . grad phi_b;
//   S4     dw/dphi_a (Eq. Obstacle / Eq. Well), psi^b(mu, T) from the parabolic
//          free energies (Sec. 3), dpsi/dphi_a = sum_b psi^b dh_b/dphi_a (Eq. hphi);
//   S5     rate of Eq. (phi_eqn) divided by tau eps, explicit Euler, and the
//          projection that realises the Lagrange multiplier;
//   S6/S7  face mobilities and the mu update of Eq. (Mu_explicit_temperature)
//          with chi(h(phi^{n+1})), c^a(mu^n), dh/dt and dT/dt as one-step
//          differences, which keeps sum_cells c conserved to round-off.
// Exactness of the bulk shortcut: a cell whose whole stencil holds a single
// phase with value exactly 1 at the centre has q = 0 for every pair, dw/dphi
// and dpsi/dphi that leave that vertex fixed under the projection, so
// phi^{n+1} = phi^n there bit for bit; only the mu update is evaluated.
#pragma once

#include <type_traits>

#include "ms_device.cuh"

namespace msgb {

// Dual-number scalars take neither the bulk shortcut nor the pair skip: both
// are exact for values but would drop derivatives (a perturbation of an absent
// phase, or of a bulk cell, has a non-zero first-order effect).
template <class S>
struct IsDual {
  static constexpr bool value = false;
};
template <class R, int W>
struct IsDual<Dual<R, W>> {
  static constexpr bool value = true;
};

// Optional parts of the cell update, as a compile-time mask: a kernel
// instantiated without one of them never takes that path (its model does not
// use it), which keeps the code and the registers of the common case small.
constexpr int kFeatRot = 1;      // rotated anisotropic pairs (Rotation_matrix)
constexpr int kFeatG3 = 2;       // the triple-junction term gamma_abc of the obstacle
constexpr int kFeatNoise = 4;    // phi noise
constexpr int kFeatElastic = 8;  // elastic potentials added to psi
constexpr int kFeatGG = 16;      // grain growth (no chemical driving force, mu held)
constexpr int kFeatSolidD = 32;  // phases other than the liquid diffuse (else M = h_l D^l chi^l)
constexpr int kFeatAll = 63;

// g = dA/dq of the unrotated anisotropic pair, evaluated in real arithmetic
// through the factorisation g_i = 2 gamma a_c q_i (a_c + 16 delta (q_i^2 /
// |q|^2 - r)), r = sum_j q_j^4 / |q|^4, a_c = (1 - 3 delta) + 4 delta r (the
// derivative of Eq. (aniso_eqn)'s A written out once), g = 0 when |q|^2 <
// 1e-12 (often the whole warp: a pair absent around it has q = 0 exactly).
// Rotated pairs and dual numbers use pair_grad.
template <int DIM, class Real>
__device__ __forceinline__ void aniso_grad_factored(const Real* q, Real gam2, Real del, Real* g,
                                                    int only = -1) {
  Real q2[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) q2[i] = q[i] * q[i];
  Real Q = q2[0], s4 = q2[0] * q2[0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) {
    Q += q2[i];
    s4 += q2[i] * q2[i];
  }
  if (Q < Real(1e-12)) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) g[i] = Real(0);
    return;
  }
  const Real invQ = recip(Q);
  const Real r = s4 * invQ * invQ;
  const Real ac = (Real(1) - Real(3) * del) + Real(4) * del * r;
  const Real ga = gam2 * ac;
  const Real k16 = Real(16) * del;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
    if (only < 0 || i == only) g[i] = ga * q[i] * (ac + k16 * (q2[i] * invQ - r));
}

// pair_grad for the forward step: the factored form for unrotated
// anisotropic pairs in real arithmetic, pair_grad otherwise.
template <int DIM, class S, class Real>
__device__ __forceinline__ void pair_grad_fwd(const S* q, Real gam2, const S& del, bool aniso, bool rotated,
                                              const Real* R, S* g) {
  if constexpr (!IsDual<S>::value) {
    if (aniso && !rotated) {
      aniso_grad_factored<DIM, Real>(q, gam2, del, g);
      return;
    }
  }
  pair_grad<DIM>(q, gam2, del, aniso, rotated, R, g);
}

// Normal component (axis D) of g_ab at a face from the face values pa, pb
// and face gradients ga, gb of the pair (q = pa gb - pb ga): isotropic pairs
// need q_D only, unrotated anisotropic ones the factored form's D component.
template <int DIM, int D, class S, class Real>
__device__ __forceinline__ S face_pair_flux(const S& pa, const S& pb, const S* ga, const S* gb, Real gam2,
                                            const S& del, bool aniso, bool rotated, const Real* R) {
  const S qD = pa * gb[D] - pb * ga[D];
  if (!aniso) return gam2 * qD;
  S q[DIM], gq[DIM];
#pragma unroll
  for (int t = 0; t < DIM; ++t) q[t] = t == D ? qD : pa * gb[t] - pb * ga[t];
  if constexpr (!IsDual<S>::value) {
    if (!rotated) {
      aniso_grad_factored<DIM, Real>(q, gam2, del, gq, D);
      return gq[D];
    }
  }
  pair_grad<DIM>(q, gam2, del, true, rotated, R, gq);
  return gq[D];
}

// Normal (axis D) component of g_ab on the two faces of a cell along D at
// once (low half: the face shared with the -D neighbour, high half: with the
// +D neighbour) in paired FP32 arithmetic: face values pa, pb, their
// negations, face gradients ga, gb.  Same forms as face_pair_flux.
template <int DIM, int D>
__device__ __forceinline__ F2 face_pair_flux2(F2 pa, F2 npb, const F2* ga, const F2* gb, float gam2, float del,
                                              bool aniso, bool rotated, const float* R) {
  const F2 qD = fma2(pa, gb[D], npb * ga[D]);
  if (!aniso) return f2s(gam2) * qD;
  F2 q[DIM];
#pragma unroll
  for (int t = 0; t < DIM; ++t) q[t] = t == D ? qD : fma2(pa, gb[t], npb * ga[t]);
  if (rotated) {
    float ql[DIM], qh[DIM], gl[DIM], gh[DIM];
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      ql[t] = f2lo(q[t]);
      qh[t] = f2hi(q[t]);
    }
    pair_grad<DIM>(ql, gam2, del, true, true, R, gl);
    pair_grad<DIM>(qh, gam2, del, true, true, R, gh);
    return f2(gl[D], gh[D]);
  }
  F2 q2[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) q2[i] = q[i] * q[i];
  F2 Q = q2[0], s4 = q2[0] * q2[0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) {
    Q = Q + q2[i];
    s4 = fma2(q2[i], q2[i], s4);
  }
  const float Ql = f2lo(Q), Qh = f2hi(Q);
  const bool tl = Ql < 1e-12f, th = Qh < 1e-12f;   // g := 0 there (selected below)
  const F2 invQ = f2(recip(tl ? 1.0f : Ql), recip(th ? 1.0f : Qh));
  const F2 r = s4 * invQ * invQ;
  const F2 ac = fma2(f2s(4.0f * del), r, f2s(1.0f - 3.0f * del));
  const F2 t = q2[D] * invQ - r;
  const F2 gD = (f2s(gam2) * ac) * qD * fma2(f2s(16.0f * del), t, ac);
  return f2(tl ? 0.0f : f2lo(gD), th ? 0.0f : f2hi(gD));
}

template <class S, int P>
struct DiffPrm {
  S mob;         // phase-field mobility 1/tau
  S delta[P];    // anisotropy strength per pair
};

template <int DIM>
struct Off {
  int x, y, z;
};

// Offset of unit step s along axis d.
template <int DIM>
__device__ __forceinline__ Off<DIM> unit(int d, int s) {
  Off<DIM> o{0, 0, 0};
  if (d == 0) o.x = s;
  if (d == 1) o.y = s;
  if (d == 2) o.z = s;
  return o;
}

template <int DIM>
__device__ __forceinline__ Off<DIM> add(Off<DIM> a, Off<DIM> b) {
  return Off<DIM>{a.x + b.x, a.y + b.y, a.z + b.z};
}

// Normal component (axis D) of J_a on one face from the face values pf and
// the face gradients gr of the phases (pairs absent from `mask` skipped).
template <int DIM, int D, int NP, int NM, class Real, class S, int FEAT = kFeatAll>
__device__ __forceinline__ void face_flux_from(const StepArgs<Real, NP, NM>& g,
                                               const DiffPrm<S, NP*(NP - 1) / 2>& dp, uint32_t mask, const S* pf,
                                               const S (*gr)[DIM], S* Jn) {
#pragma unroll
  for (int a = 0; a < NP; ++a) Jn[a] = S(Real(0));
  int p = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b, ++p) {
      if (!(((mask >> a) & (mask >> b)) & 1u)) continue;
      const S gD = face_pair_flux<DIM, D>(pf[a], pf[b], gr[a], gr[b], g.gam2[p], dp.delta[p], g.aniso[p] != 0,
                                          (FEAT & kFeatRot) && g.rotated[p] != 0, g.rot[p]);
      Jn[a] -= pf[b] * gD;
      Jn[b] += pf[a] * gD;
    }
  }
}

// Normal component (axis D) of J_a on one face of the cell: side 0 = the
// face shared with the -D neighbour, side 1 = with the +D neighbour.
template <int DIM, int D, int NP, int NM, class Real, class S, class Acc, int FEAT = kFeatAll>
__device__ __forceinline__ void face_flux(const Acc& A, const StepArgs<Real, NP, NM>& g,
                                          const DiffPrm<S, NP*(NP - 1) / 2>& dp, uint32_t mask,
                                          int side, bool need_tan, S* Jn) {
  const Off<DIM> L = unit<DIM>(D, side ? 0 : -1);
  const Off<DIM> R = unit<DIM>(D, side ? 1 : 0);
  S pf[NP];
  S gr[NP][DIM];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    if (!((mask >> a) & 1u)) continue;
    S vl = A.phi(a, L.x, L.y, L.z);
    S vr = A.phi(a, R.x, R.y, R.z);
    pf[a] = Real(0.5) * (vl + vr);
    gr[a][D] = (vr - vl) * g.inv_dx;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == D) continue;
      if (need_tan) {
        const Off<DIM> up = unit<DIM>(t, 1), dn = unit<DIM>(t, -1);
        const Off<DIM> Lu = add(L, up), Ru = add(R, up), Ld = add(L, dn), Rd = add(R, dn);
        gr[a][t] = ((A.phi(a, Lu.x, Lu.y, Lu.z) + A.phi(a, Ru.x, Ru.y, Ru.z)) -
                    (A.phi(a, Ld.x, Ld.y, Ld.z) + A.phi(a, Rd.x, Rd.y, Rd.z))) *
                   g.quarter_inv_dx;
      } else {
        gr[a][t] = S(Real(0));
      }
    }
  }
  face_flux_from<DIM, D, NP, NM, Real, S, FEAT>(g, dp, mask, pf, gr, Jn);
}

// Both faces along axis D at once in paired FP32 arithmetic (low half: the
// face with the -D neighbour, high half: with the +D neighbour); the same
// discretisation as face_flux, J[a] = (J_a on the low face, on the high face).
template <int DIM, int D, int NP, int NM, class Acc, int FEAT = kFeatAll, bool ALL = false>
__device__ __forceinline__ void face_flux_pair(const Acc& A, const StepArgs<float, NP, NM>& g, uint32_t mask,
                                               bool need_tan, const float (*gcr)[DIM], F2* J) {
  const Off<DIM> m = unit<DIM>(D, -1), p = unit<DIM>(D, 1);
  F2 pf[NP], npf[NP], gr[NP][DIM];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    J[a] = f2s(0.0f);
    if (!ALL && !((mask >> a) & 1u)) continue;
    const float vm = A.phi(a, m.x, m.y, m.z), v0 = A.phi(a, 0, 0, 0), vp = A.phi(a, p.x, p.y, p.z);
    const F2 vl = f2(vm, v0), vr = f2(v0, vp);
    pf[a] = f2s(0.5f) * (vl + vr);
    npf[a] = f2s(-0.5f) * (vl + vr);
    gr[a][D] = (vr - vl) * f2s(g.inv_dx);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == D) continue;
      if (ALL || need_tan) {
        // the 4-point average (1/4)[(L+t) + (R+t) - (L-t) - (R-t)] written as
        // the sum of the two cells' central differences along t: the
        // neighbours' from the edge values, the cell's own (gcr) shared with
        // the centre term
        const Off<DIM> up = unit<DIM>(t, 1), dn = unit<DIM>(t, -1);
        const Off<DIM> mu_ = add(m, up), md = add(m, dn), pu = add(p, up), pd = add(p, dn);
        const F2 nb = f2(A.phi(a, mu_.x, mu_.y, mu_.z), A.phi(a, pu.x, pu.y, pu.z)) -
                      f2(A.phi(a, md.x, md.y, md.z), A.phi(a, pd.x, pd.y, pd.z));
        gr[a][t] = (nb + f2s(gcr[a][t])) * f2s(g.quarter_inv_dx);
      } else {
        gr[a][t] = f2s(0.0f);
      }
    }
  }
  int pi = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b, ++pi) {
      if (!ALL && !(((mask >> a) & (mask >> b)) & 1u)) continue;
      const F2 gD = face_pair_flux2<DIM, D>(pf[a], npf[b], gr[a], gr[b], g.gam2[pi], g.delta[pi], g.aniso[pi] != 0,
                                            (FEAT & kFeatRot) && g.rotated[pi] != 0, g.rot[pi]);
      J[a] = fma2(npf[b], gD, J[a]);
      J[b] = fma2(pf[a], gD, J[b]);
    }
  }
}

// Cell mobilities M = sum_a h_a D^a chi^a of the two neighbours along axis d
// at once (low half: the -d neighbour, high half: the +d one), paired FP32.
template <int DIM, int NP, int NM, class Acc>
__device__ __forceinline__ void mobility_pair(const Acc& A, const StepArgs<float, NP, NM>& g, int d, F2* M) {
  const Off<DIM> m = unit<DIM>(d, -1), p = unit<DIM>(d, 1);
  F2 f[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) f[a] = f2(A.phi(a, m.x, m.y, m.z), A.phi(a, p.x, p.y, p.z));
  F2 e1 = f[0], e2 = f2s(0.0f), run = f[0];
#pragma unroll
  for (int a = 1; a < NP; ++a) {
    e1 = e1 + f[a];
    e2 = fma2(f[a], run, e2);
    run = run + f[a];
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const F2 rest = e2 - f[a] * (e1 - f[a]);
    const F2 p2 = f[a] * f[a];
    const F2 h = f2s(3.0f) * p2 - f2s(2.0f) * p2 * f[a] + f2s(2.0f) * f[a] * rest;
#pragma unroll
    for (int k = 0; k < NM * NM; ++k) M[k] = a == 0 ? h * f2s(g.DX[0][k]) : fma2(h, f2s(g.DX[a][k]), M[k]);
  }
}

// As mobility_pair when only the liquid (phase NP-1) diffuses: M = h_l D^l
// chi^l, h_l = phi_l^2 (3 - 2 phi_l) + 2 phi_l sum_{b<c<l} phi_b phi_c.
template <int DIM, int NP, int NM, class Acc>
__device__ __forceinline__ void mobility_pair_liquid(const Acc& A, const StepArgs<float, NP, NM>& g, int d, F2* M) {
  const Off<DIM> m = unit<DIM>(d, -1), p = unit<DIM>(d, 1);
  constexpr int L = NP - 1;
  F2 f[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) f[a] = f2(A.phi(a, m.x, m.y, m.z), A.phi(a, p.x, p.y, p.z));
  F2 rest = f2s(0.0f), run = f[0];
#pragma unroll
  for (int b = 1; b < L; ++b) {
    rest = fma2(f[b], run, rest);
    run = run + f[b];
  }
  const F2 p2 = f[L] * f[L];
  const F2 h = f2s(3.0f) * p2 - f2s(2.0f) * p2 * f[L] + f2s(2.0f) * f[L] * rest;
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) M[k] = h * f2s(g.DX[L][k]);
}

// The cell's own mobility when only the liquid diffuses (scalar).
template <int NP, int NM, class Real>
__device__ __forceinline__ void mobility_liquid(const Real* ph, const StepArgs<Real, NP, NM>& g, Real* M) {
  constexpr int L = NP - 1;
  Real rest = Real(0), run = ph[0];
#pragma unroll
  for (int b = 1; b < L; ++b) {
    rest += ph[b] * run;
    run += ph[b];
  }
  const Real p2 = ph[L] * ph[L];
  const Real h = Real(3) * p2 - Real(2) * p2 * ph[L] + Real(2) * ph[L] * rest;
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) M[k] = h * g.DX[L][k];
}

// psi^b(mu, T) = C^b(T) - 1/2 (mu - B^b)^T chi^b (mu - B^b), s = T - T_ref.
template <int NP, int NM, class Real, class S>
__device__ __forceinline__ S grand_potential(const StepArgs<Real, NP, NM>& g, int b, const S* mu,
                                             Real s) {
  S y[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) y[j] = mu[j] - (g.B0[b][j] + g.B1[b][j] * s);
  S quad = S(Real(0));
#pragma unroll
  for (int i = 0; i < NM; ++i) {
#pragma unroll
    for (int j = 0; j < NM; ++j) quad += y[i] * (g.chi[b][i * NM + j] * y[j]);
  }
  const Real C = g.C0[b] + s * (g.C1[b] + s * g.C2[b]);
  return C - Real(0.5) * quad;
}

// Centre term of S3, Gc_a = sum_b g_ab . grad phi_b (with the opposite sign
// for b), from the unscaled central differences gcr of the phases and the
// cell's own phi.
template <int DIM, int NP, int NM, class Real, class S, int FEAT, bool ALL>
__device__ __forceinline__ void centre_term(const StepArgs<Real, NP, NM>& g, const DiffPrm<S, NP*(NP - 1) / 2>& dp,
                                            const S* ph, const S (*gcr)[DIM], uint32_t mask, S* Gc) {
  S gc[NP][DIM];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    if (!ALL && !((mask >> a) & 1u)) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) gc[a][d] = S(Real(0));
      continue;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) gc[a][d] = gcr[a][d] * g.half_inv_dx;
  }
  int p = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b, ++p) {
      if (!ALL && !(((mask >> a) & (mask >> b)) & 1u)) continue;
      S q[DIM], gq[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) q[d] = ph[a] * gc[b][d] - ph[b] * gc[a][d];
      pair_grad_fwd<DIM>(q, g.gam2[p], dp.delta[p], g.aniso[p] != 0, (FEAT & kFeatRot) && g.rotated[p] != 0,
                         g.rot[p], gq);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        Gc[a] += gq[d] * gc[b][d];
        Gc[b] -= gq[d] * gc[a][d];
      }
    }
  }
}

// S1-S3 of the cell update: divergence of the face fluxes and the centre
// term.  ALL: every phase is present in the stencil region and some present
// pair is anisotropic (the row's mask says so), so no per-phase or per-pair
// test is needed and the code is straight-line.
template <int DIM, int NP, int NM, class Real, class S, class Acc, int FEAT, bool ALL>
__device__ __forceinline__ void gradient_terms(const Acc& A, const StepArgs<Real, NP, NM>& g,
                                               const DiffPrm<S, NP*(NP - 1) / 2>& dp, const S* ph, uint32_t mask,
                                               bool need_tan, S* divJ, S* Gc) {
  // central differences (unscaled) of the present phases: the centre
  // term and, in FP32, the tangential face gradients
  S gcr[NP][DIM];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    if (!ALL && !((mask >> a) & 1u)) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) gcr[a][d] = S(Real(0));
      continue;
    }
    gcr[a][0] = A.phi(a, 1, 0, 0) - A.phi(a, -1, 0, 0);
    gcr[a][1] = A.phi(a, 0, 1, 0) - A.phi(a, 0, -1, 0);
    if constexpr (DIM == 3) gcr[a][2] = A.phi(a, 0, 0, 1) - A.phi(a, 0, 0, -1);
  }
  // S1-S3: divergence of the face fluxes
  {
    if constexpr (std::is_same<S, float>::value) {
      F2 J[NP];
      face_flux_pair<DIM, 0, NP, NM, Acc, FEAT, ALL>(A, g, mask, need_tan, gcr, J);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (f2hi(J[a]) - f2lo(J[a])) * g.inv_dx;
    } else {
      S Jm[NP], Jp[NP];
      face_flux<DIM, 0, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 0, need_tan, Jm);
      face_flux<DIM, 0, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 1, need_tan, Jp);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (Jp[a] - Jm[a]) * g.inv_dx;
    }
  }
  {
    if constexpr (std::is_same<S, float>::value) {
      F2 J[NP];
      face_flux_pair<DIM, 1, NP, NM, Acc, FEAT, ALL>(A, g, mask, need_tan, gcr, J);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (f2hi(J[a]) - f2lo(J[a])) * g.inv_dx;
    } else {
      S Jm[NP], Jp[NP];
      face_flux<DIM, 1, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 0, need_tan, Jm);
      face_flux<DIM, 1, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 1, need_tan, Jp);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (Jp[a] - Jm[a]) * g.inv_dx;
    }
  }
  if constexpr (DIM == 3) {
    if constexpr (std::is_same<S, float>::value) {
      F2 J[NP];
      face_flux_pair<DIM, 2, NP, NM, Acc, FEAT, ALL>(A, g, mask, need_tan, gcr, J);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (f2hi(J[a]) - f2lo(J[a])) * g.inv_dx;
    } else {
      S Jm[NP], Jp[NP];
      face_flux<DIM, 2, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 0, need_tan, Jm);
      face_flux<DIM, 2, NP, NM, Real, S, Acc, FEAT>(A, g, dp, mask, 1, need_tan, Jp);
#pragma unroll
      for (int a = 0; a < NP; ++a) divJ[a] += (Jp[a] - Jm[a]) * g.inv_dx;
    }
  }
  centre_term<DIM, NP, NM, Real, S, FEAT, ALL>(g, dp, ph, gcr, mask, Gc);
}

// S4-S5 of the cell update from the gradient terms: the potential
// derivative, the driving force, the rate of Eq. (phi_eqn) / (tau eps), the
// explicit Euler step and the projection.  ph, mc: the cell's phi^n and mu^n;
// divJ, Gc: divergence of the face fluxes and the centre term; s = T - T_ref.
template <int DIM, int NP, int NM, class Real, class S, int FEAT = kFeatAll>
__device__ __forceinline__ void phase_update(const StepArgs<Real, NP, NM>& g, const DiffPrm<S, NP*(NP - 1) / 2>& dp,
                                             const S* ph, const S* mc, const S* divJ, const S* Gc, Real s,
                                             unsigned long long gcell, S* pn) {
  const bool gg = (FEAT & kFeatGG) && g.gg;
  // S4: potential derivative
  S W[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    W[a] = S(Real(0));
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      if (b == a) continue;
      if (g.potential == 1)
        W[a] += g.cw[a][b] * ph[b];
      else
        W[a] += g.cw[a][b] * (ph[a] * (ph[b] * ph[b]));
    }
    if ((FEAT & kFeatG3) && g.has_g3) {
#pragma unroll
      for (int b = 0; b < NP; ++b)
#pragma unroll
        for (int e = b + 1; e < NP; ++e)
          if (b != a && e != a) W[a] += g.g3[a][b][e] * (ph[b] * ph[e]);
    }
  }
  // S4: driving force sum_b psi^b dh_b/dphi_a
  S psi[NP];
#pragma unroll
  for (int b = 0; b < NP; ++b) psi[b] = gg ? S(Real(0)) : grand_potential<NP, NM, Real>(g, b, mc, s);
  if ((FEAT & kFeatElastic) && g.elw) {   // elasticity: -sigma : eps*^b joins each phase potential
    const unsigned long long cell = gcell - (unsigned long long)g.zorg * (DIM == 3 ? (unsigned long long)g.nx * g.ny : g.nx);
    const unsigned long long cells = (unsigned long long)g.nx * g.ny * (DIM == 3 ? g.nz : 1);
#pragma unroll
    for (int b = 0; b < NP; ++b) psi[b] = psi[b] + g.elw[b * cells + cell];
  }
  S e1 = ph[0];
#pragma unroll
  for (int a = 1; a < NP; ++a) e1 += ph[a];
  S e2 = S(Real(0));
  {
    S run = ph[0];
#pragma unroll
    for (int a = 1; a < NP; ++a) {
      e2 += ph[a] * run;
      run += ph[a];
    }
  }
  S v[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    S rest = e2 - ph[a] * (e1 - ph[a]);
    S P = psi[a] * (Real(6) * ph[a] - Real(6) * (ph[a] * ph[a]) + Real(2) * rest);
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      if (b == a) continue;
      P += psi[b] * (Real(2) * ph[b] * ((e1 - ph[a]) - ph[b]));
    }
    // S5: rate of Eq. (phi_eqn) / (tau eps), explicit Euler
    S r = dp.mob * ((g.eps * (divJ[a] - Gc[a]) - W[a] * g.inv_eps - P) * g.inv_eps);
    v[a] = ph[a] + g.dt * r;
    // phi noise on the interface phases of the cell (0 < phi_a < 1)
    if ((FEAT & kFeatNoise) && g.noise_amp != Real(0) && val(ph[a]) > Real(0) && val(ph[a]) < Real(1))
      v[a] = v[a] + g.dt * g.noise_amp * noise_variate<Real>(g.noise_seed, g.step, gcell * NP + a);
  }
  project<NP>(g.potential, v, pn);
}

// S7 of the cell update from the flux divergence div = sum_faces M_f grad mu:
// the mu step of Eq. (Mu_explicit_temperature) with chi(h(phi^{n+1})),
// c^a(mu^n) and dh/dt, dT/dt as one-step differences.  bulk: phi^{n+1} =
// phi^n (no dh term).
template <int NP, int NM, class Real, class S>
__device__ __forceinline__ void mu_update(const StepArgs<Real, NP, NM>& g, const S* ph, const S* pn, const S* mc,
                                          const S* div, Real s, bool bulk, S* mn) {
  S h_new[NP];
  interp_h<NP>(pn, h_new);
  S rhs[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) rhs[i] = g.dt * div[i];
  if (!bulk) {
    S h_old[NP];
    interp_h<NP>(ph, h_old);
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      S dh = h_new[a] - h_old[a];
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        S c_now = S(Real(0));
#pragma unroll
        for (int j = 0; j < NM; ++j)
          c_now += g.chi[a][i * NM + j] * (mc[j] - (g.B0[a][j] + g.B1[a][j] * s));
        rhs[i] -= c_now * dh;
        rhs[i] -= h_new[a] * g.dcT[a][i];
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a)
#pragma unroll
      for (int i = 0; i < NM; ++i) rhs[i] -= h_new[a] * g.dcT[a][i];
  }
  S chi[NM * NM];
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) {
    chi[k] = h_new[0] * g.chi[0][k];
#pragma unroll
    for (int a = 1; a < NP; ++a) chi[k] += h_new[a] * g.chi[a][k];
  }
  S dmu[NM];
  solve_small<NM>(chi, rhs, dmu);
#pragma unroll
  for (int i = 0; i < NM; ++i) mn[i] = mc[i] + dmu[i];
}

// The full cell update.  kz = cell index along the last axis (for T).
template <int DIM, int NP, int NM, class Real, class S, class Acc, int FEAT = kFeatAll>
__device__ __forceinline__ void gp_cell(const Acc& A, const StepArgs<Real, NP, NM>& g,
                                        const DiffPrm<S, NP*(NP - 1) / 2>& dp, int kz, unsigned long long gcell,
                                        S* pn, S* mn) {
  const bool gg = (FEAT & kFeatGG) && g.gg;
  S ph[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) ph[a] = A.phi(a, 0, 0, 0);
  const uint32_t mask = A.mask();
  const int npresent = __popc(mask);
  bool bulk = false;
  if (!IsDual<S>::value && npresent == 1) {
    const int l = __ffs(mask) - 1;
#pragma unroll
    for (int a = 0; a < NP; ++a)
      if (a == l) bulk = (val(ph[a]) == Real(1));
  }
  const Real s = g.tz0 + g.tzg * (Real(kz) + Real(0.5));   // T^n - T_ref
  S mc[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mc[i] = A.mu(i, 0, 0, 0);

  if (bulk) {
#pragma unroll
    for (int a = 0; a < NP; ++a) pn[a] = ph[a];
  } else {
    S divJ[NP], Gc[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      divJ[a] = S(Real(0));
      Gc[a] = S(Real(0));
    }
    if (npresent >= 2) {
      bool need_tan = false;
      {
        int p = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a)
#pragma unroll
          for (int b = a + 1; b < NP; ++b, ++p)
            if ((((mask >> a) & (mask >> b)) & 1u) && g.aniso[p]) need_tan = true;
      }
      if constexpr (std::is_same<S, float>::value) {
        if (mask == (1u << NP) - 1u && need_tan)
          gradient_terms<DIM, NP, NM, Real, S, Acc, FEAT, true>(A, g, dp, ph, mask, need_tan, divJ, Gc);
        else
          gradient_terms<DIM, NP, NM, Real, S, Acc, FEAT, false>(A, g, dp, ph, mask, need_tan, divJ, Gc);
      } else {
        gradient_terms<DIM, NP, NM, Real, S, Acc, FEAT, false>(A, g, dp, ph, mask, need_tan, divJ, Gc);
      }
    }
    phase_update<DIM, NP, NM, Real, S, FEAT>(g, dp, ph, mc, divJ, Gc, s, gcell, pn);
  }
  if (gg) {   // grain growth: mu held
#pragma unroll
    for (int i = 0; i < NM; ++i) mn[i] = mc[i];
    return;
  }

  // ---- S6/S7: chemical-potential update
  S Mc[NM * NM];
  if constexpr (!(FEAT & kFeatSolidD) && std::is_same<S, Real>::value) {
    S phc[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) phc[a] = A.phi(a, 0, 0, 0);
    mobility_liquid<NP, NM, Real>(phc, g, Mc);
  } else {
    A.mobility(0, 0, 0, Mc);
  }
  S div[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) div[i] = S(Real(0));
  if constexpr (std::is_same<S, float>::value) {
    // both neighbours along each axis at once (paired FP32)
    F2 dv[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) dv[i] = f2s(0.0f);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const Off<DIM> m = unit<DIM>(d, -1), p = unit<DIM>(d, 1);
      F2 Mn[NM * NM];
      if constexpr (FEAT & kFeatSolidD)
        mobility_pair<DIM, NP, NM>(A, g, d, Mn);
      else
        mobility_pair_liquid<DIM, NP, NM>(A, g, d, Mn);
#pragma unroll
      for (int i = 0; i < NM; ++i) {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          const F2 Mf = f2s(0.5f) * (f2s(Mc[i * NM + j]) + Mn[i * NM + j]);
          const F2 dm = f2(A.mu(j, m.x, m.y, m.z), A.mu(j, p.x, p.y, p.z)) - f2s(mc[j]);
          dv[i] = fma2(Mf, dm * f2s(g.inv_dx2), dv[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) div[i] = f2lo(dv[i]) + f2hi(dv[i]);
  } else {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int sd = -1; sd <= 1; sd += 2) {
        const Off<DIM> o = unit<DIM>(d, sd);
        S Mn[NM * NM];
        A.mobility(o.x, o.y, o.z, Mn);
#pragma unroll
        for (int i = 0; i < NM; ++i) {
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            S Mf = Real(0.5) * (Mc[i * NM + j] + Mn[i * NM + j]);
            div[i] += Mf * ((A.mu(j, o.x, o.y, o.z) - mc[j]) * g.inv_dx2);
          }
        }
      }
    }
  }
  mu_update<NP, NM, Real, S>(g, ph, pn, mc, div, s, bulk, mn);
}

// ------------------------------------------------------------------------
// The same update for many phases, when the phase mask (uniform over the
// warp; a superset of every cell's stencil) names at most KP phases: the
// gradient work -- face fluxes, centre term, face mobilities -- runs on the
// compact list of present phases; the potential, driving force, rates and the
// projection run over all NP phases (an absent phase has phi = 0 on the whole
// stencil, so every gradient term it would enter is exactly zero, but its
// rate need not be).  Sums keep the order of gp_cell over the non-zero terms.
// Real arithmetic only (the adjoint's dual numbers use gp_cell).

// Normal face fluxes of the present phases on one face (compact index k).
template <int DIM, int D, int NP, int NM, int KP, class Real, class Acc, int FEAT = kFeatAll>
__device__ __forceinline__ void face_flux_sparse(const Acc& A, const StepArgs<Real, NP, NM>& g, const int* map,
                                                 int kn, int side, bool need_tan, Real* Jk) {
  const Off<DIM> L = unit<DIM>(D, side ? 0 : -1);
  const Off<DIM> R = unit<DIM>(D, side ? 1 : 0);
  Real pf[KP], gr[KP][DIM];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    Jk[k] = Real(0);
    if (k >= kn) continue;
    const int a = map[k];
    const Real vl = A.phi(a, L.x, L.y, L.z), vr = A.phi(a, R.x, R.y, R.z);
    pf[k] = Real(0.5) * (vl + vr);
    gr[k][D] = (vr - vl) * g.inv_dx;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == D) continue;
      if (need_tan) {
        const Off<DIM> up = unit<DIM>(t, 1), dn = unit<DIM>(t, -1);
        const Off<DIM> Lu = add(L, up), Ru = add(R, up), Ld = add(L, dn), Rd = add(R, dn);
        gr[k][t] = ((A.phi(a, Lu.x, Lu.y, Lu.z) + A.phi(a, Ru.x, Ru.y, Ru.z)) -
                    (A.phi(a, Ld.x, Ld.y, Ld.z) + A.phi(a, Rd.x, Rd.y, Rd.z))) *
                   g.quarter_inv_dx;
      } else {
        gr[k][t] = Real(0);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KP; ++k) {
#pragma unroll
    for (int l = k + 1; l < KP; ++l) {
      if (l >= kn) continue;
      const int p = pair_index<NP>(map[k], map[l]);
      const Real gD = face_pair_flux<DIM, D>(pf[k], pf[l], gr[k], gr[l], g.gam2[p], g.delta[p], g.aniso[p] != 0,
                                             (FEAT & kFeatRot) && g.rotated[p] != 0, g.rot[p]);
      Jk[k] -= pf[l] * gD;
      Jk[l] += pf[k] * gD;
    }
  }
}

// Cell mobility of a stencil cell from the present phases only (the absent
// ones have h = 0 there): e1, e2 and the sum over phases as in cell_mobility.
template <int DIM, int NP, int NM, int KP, class Real, class Acc>
__device__ __forceinline__ void mobility_sparse(const Acc& A, const StepArgs<Real, NP, NM>& g, const int* map,
                                                int kn, int dx, int dy, int dz, Real* M) {
  Real f[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) f[k] = k < kn ? A.phi(map[k], dx, dy, dz) : Real(0);
  Real e1 = f[0];
#pragma unroll
  for (int k = 1; k < KP; ++k) e1 += f[k];
  Real e2 = Real(0);
  {
    Real run = f[0];
#pragma unroll
    for (int k = 1; k < KP; ++k) {
      e2 += f[k] * run;
      run += f[k];
    }
  }
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    if (k >= kn) break;
    const Real rest = e2 - f[k] * (e1 - f[k]);
    const Real p2 = f[k] * f[k];
    const Real h = Real(3) * p2 - Real(2) * p2 * f[k] + Real(2) * f[k] * rest;
    const int a = map[k];
#pragma unroll
    for (int q = 0; q < NM * NM; ++q) M[q] = k == 0 ? h * g.DX[a][q] : M[q] + h * g.DX[a][q];
  }
}

template <int DIM, int NP, int NM, int KP, class Real, class Acc, int FEAT = kFeatAll>
__device__ __forceinline__ void gp_cell_sparse(const Acc& A, const StepArgs<Real, NP, NM>& g, int kz,
                                               unsigned long long gcell, Real* pn, Real* mn) {
  const bool gg = (FEAT & kFeatGG) && g.gg;
  static_assert(!IsDual<Real>::value, "real arithmetic only");
  const uint32_t mask = A.mask();
  const int kn = __popc(mask);
  int map[KP];   // present phases, increasing
  {
    uint32_t m = mask;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      map[k] = m ? __ffs(m) - 1 : 0;
      m &= m - 1u;
    }
  }
  Real ph[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) ph[a] = ((mask >> a) & 1u) ? A.phi(a, 0, 0, 0) : Real(0);
  const bool bulk = kn == 1 && A.phi(map[0], 0, 0, 0) == Real(1);
  const Real s = g.tz0 + g.tzg * (Real(kz) + Real(0.5));   // T^n - T_ref
  Real mc[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mc[i] = A.mu(i, 0, 0, 0);

  if (bulk) {
#pragma unroll
    for (int a = 0; a < NP; ++a) pn[a] = ph[a];
  } else {
    Real dg[KP];   // divJ - Gc of the present phases
#pragma unroll
    for (int k = 0; k < KP; ++k) dg[k] = Real(0);
    if (kn >= 2) {
      bool need_tan = false;
#pragma unroll
      for (int k = 0; k < KP; ++k)
#pragma unroll
        for (int l = k + 1; l < KP; ++l)
          if (l < kn && g.aniso[pair_index<NP>(map[k], map[l])]) need_tan = true;
      Real divJ[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) divJ[k] = Real(0);
      {
        Real Jm[KP], Jp[KP];
        face_flux_sparse<DIM, 0, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 0, need_tan, Jm);
        face_flux_sparse<DIM, 0, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 1, need_tan, Jp);
#pragma unroll
        for (int k = 0; k < KP; ++k) divJ[k] += (Jp[k] - Jm[k]) * g.inv_dx;
      }
      {
        Real Jm[KP], Jp[KP];
        face_flux_sparse<DIM, 1, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 0, need_tan, Jm);
        face_flux_sparse<DIM, 1, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 1, need_tan, Jp);
#pragma unroll
        for (int k = 0; k < KP; ++k) divJ[k] += (Jp[k] - Jm[k]) * g.inv_dx;
      }
      if constexpr (DIM == 3) {
        Real Jm[KP], Jp[KP];
        face_flux_sparse<DIM, 2, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 0, need_tan, Jm);
        face_flux_sparse<DIM, 2, NP, NM, KP, Real, Acc, FEAT>(A, g, map, kn, 1, need_tan, Jp);
#pragma unroll
        for (int k = 0; k < KP; ++k) divJ[k] += (Jp[k] - Jm[k]) * g.inv_dx;
      }
      // centre term, central differences
      Real gc[KP][DIM], Gc[KP], phk[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        Gc[k] = Real(0);
        phk[k] = k < kn ? A.phi(map[k], 0, 0, 0) : Real(0);
        if (k >= kn) continue;
        const int a = map[k];
        gc[k][0] = (A.phi(a, 1, 0, 0) - A.phi(a, -1, 0, 0)) * g.half_inv_dx;
        gc[k][1] = (A.phi(a, 0, 1, 0) - A.phi(a, 0, -1, 0)) * g.half_inv_dx;
        if constexpr (DIM == 3) gc[k][2] = (A.phi(a, 0, 0, 1) - A.phi(a, 0, 0, -1)) * g.half_inv_dx;
      }
#pragma unroll
      for (int k = 0; k < KP; ++k) {
#pragma unroll
        for (int l = k + 1; l < KP; ++l) {
          if (l >= kn) continue;
          const int p = pair_index<NP>(map[k], map[l]);
          Real q[DIM], gq[DIM];
#pragma unroll
          for (int d = 0; d < DIM; ++d) q[d] = phk[k] * gc[l][d] - phk[l] * gc[k][d];
          pair_grad_fwd<DIM>(q, g.gam2[p], g.delta[p], g.aniso[p] != 0, (FEAT & kFeatRot) && g.rotated[p] != 0,
                             g.rot[p], gq);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            Gc[k] += gq[d] * gc[l][d];
            Gc[l] -= gq[d] * gc[k][d];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < KP; ++k) dg[k] = divJ[k] - Gc[k];
    }
    // S4: potential derivative over all phases, sums over the present ones
    Real W[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      W[a] = Real(0);
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        if (k >= kn || map[k] == a) continue;
        const int b = map[k];
        if (g.potential == 1)
          W[a] += g.cw[a][b] * ph[b];
        else
          W[a] += g.cw[a][b] * (ph[a] * (ph[b] * ph[b]));
      }
      if ((FEAT & kFeatG3) && g.has_g3) {
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int l = k + 1; l < KP; ++l)
            if (l < kn && map[k] != a && map[l] != a) W[a] += g.g3[a][map[k]][map[l]] * (ph[map[k]] * ph[map[l]]);
      }
    }
    // S4: driving force
    Real psi[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) psi[b] = gg ? Real(0) : grand_potential<NP, NM, Real>(g, b, mc, s);
    if ((FEAT & kFeatElastic) && g.elw) {   // elasticity: -sigma : eps*^b joins each phase potential
      const unsigned long long cell = gcell - (unsigned long long)g.zorg * (DIM == 3 ? (unsigned long long)g.nx * g.ny : g.nx);
      const unsigned long long cells = (unsigned long long)g.nx * g.ny * (DIM == 3 ? g.nz : 1);
#pragma unroll
      for (int b = 0; b < NP; ++b) psi[b] += g.elw[b * cells + cell];
    }
    Real e1 = ph[0];
#pragma unroll
    for (int a = 1; a < NP; ++a) e1 += ph[a];
    Real e2 = Real(0);
    {
      Real run = ph[0];
#pragma unroll
      for (int a = 1; a < NP; ++a) {
        e2 += ph[a] * run;
        run += ph[a];
      }
    }
    Real v[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      Real rest = e2 - ph[a] * (e1 - ph[a]);
      Real P = psi[a] * (Real(6) * ph[a] - Real(6) * (ph[a] * ph[a]) + Real(2) * rest);
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        if (k >= kn || map[k] == a) continue;
        const int b = map[k];
        P += psi[b] * (Real(2) * ph[b] * ((e1 - ph[a]) - ph[b]));
      }
      Real d = Real(0);
#pragma unroll
      for (int k = 0; k < KP; ++k)
        if (k < kn && map[k] == a) d = dg[k];
      // S5: rate of Eq. (phi_eqn) / (tau eps), explicit Euler
      Real r = g.mob * ((g.eps * d - W[a] * g.inv_eps - P) * g.inv_eps);
      v[a] = ph[a] + g.dt * r;
      if ((FEAT & kFeatNoise) && g.noise_amp != Real(0) && ph[a] > Real(0) && ph[a] < Real(1))
        v[a] = v[a] + g.dt * g.noise_amp * noise_variate<Real>(g.noise_seed, g.step, gcell * NP + a);
    }
    project<NP>(g.potential, v, pn);
  }
  if (gg) {   // grain growth: mu held
#pragma unroll
    for (int i = 0; i < NM; ++i) mn[i] = mc[i];
    return;
  }

  // ---- S6/S7: chemical-potential update (mobilities from the present phases)
  Real h_new[NP];
  interp_h<NP>(pn, h_new);
  Real Mc[NM * NM];
  mobility_sparse<DIM, NP, NM, KP>(A, g, map, kn, 0, 0, 0, Mc);
  Real div[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) div[i] = Real(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
#pragma unroll
    for (int sd = -1; sd <= 1; sd += 2) {
      const Off<DIM> o = unit<DIM>(d, sd);
      Real Mn[NM * NM];
      mobility_sparse<DIM, NP, NM, KP>(A, g, map, kn, o.x, o.y, o.z, Mn);
#pragma unroll
      for (int i = 0; i < NM; ++i) {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          Real Mf = Real(0.5) * (Mc[i * NM + j] + Mn[i * NM + j]);
          div[i] += Mf * ((A.mu(j, o.x, o.y, o.z) - mc[j]) * g.inv_dx2);
        }
      }
    }
  }
  Real rhs[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) rhs[i] = g.dt * div[i];
  if (!bulk) {
    Real h_old[NP];
    interp_h<NP>(ph, h_old);
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      Real dh = h_new[a] - h_old[a];
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        Real c_now = Real(0);
#pragma unroll
        for (int j = 0; j < NM; ++j) c_now += g.chi[a][i * NM + j] * (mc[j] - (g.B0[a][j] + g.B1[a][j] * s));
        rhs[i] -= c_now * dh;
        rhs[i] -= h_new[a] * g.dcT[a][i];
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a)
#pragma unroll
      for (int i = 0; i < NM; ++i) rhs[i] -= h_new[a] * g.dcT[a][i];
  }
  Real chi[NM * NM];
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) {
    chi[k] = h_new[0] * g.chi[0][k];
#pragma unroll
    for (int a = 1; a < NP; ++a) chi[k] += h_new[a] * g.chi[a][k];
  }
  Real dmu[NM];
  solve_small<NM>(chi, rhs, dmu);
#pragma unroll
  for (int i = 0; i < NM; ++i) mn[i] = mc[i] + dmu[i];
}

}  // namespace msgb
