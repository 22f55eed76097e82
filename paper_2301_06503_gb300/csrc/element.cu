// Element integration and deterministic assembly of the LGDM coupled system.
//
// element_kernel: one team of NEN threads per element (NEN = NGP for the
// 2-node bar, 4-node quad and 8-node hex with 2/2x2/2x2x2 Gauss rules, and
// for the mixed-order 3-node bar and 9-node quad with 3/3x3 rules).
//   Phase 1: thread q evaluates Gauss point q of its element: Jacobian,
//     shape derivatives, strain (B_u u), micro-equivalent strain and its
//     gradient, modified von Mises equivalent strain and gradient (Eq. A.3),
//     trial history kappa = max(kappa_hist, ebar) (Eq. A.2), damage D and
//     dD/dkappa (Eq. A.1), interaction g and dg/dD (Eq. A.4), stresses
//     (Eq. 2 without its h-term, Eq. 3-4), and stores the per-point factors
//     the element matrices need in shared memory.
//   Phase 2: thread a forms block row a of the element tangent (Eq. 11a-d)
//     and of the residual r = -F (Eq. 11e-f) by summing over the Gauss
//     points; the element matrix goes to a scratch buffer in node-block
//     layout Ke[e][a][i][b][j].
// gather_kernel: one thread per node pair (a, b) sums the nd x nd blocks of
//   every element containing both nodes, in the fixed order of a
//   precomputed contribution list (no float atomics), applies identity
//   rows / zero columns on Dirichlet dofs and writes the CSR values; the
//   diagonal pairs also sum the residual.
#include "lgdm_internal.cuh"
#include "node_block.cuh"
#include <cmath>

namespace lgdm {

MatConst make_matconst(const lgdm_material &m, int dim) {
  MatConst c{};
  if (dim == 1) {
    c.lam = m.E;
    c.mu = 0.0;
  } else {
    c.lam = m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu));
    c.mu = m.E / (2.0 * (1.0 + m.nu));
  }
  c.evm_a = (m.k - 1.0) / (2.0 * m.k * (1.0 - 2.0 * m.nu));
  const double b = (m.k - 1.0) / (1.0 - 2.0 * m.nu);
  c.evm_b2 = b * b;
  c.evm_cJ = (m.evm_variant == 0) ? 12.0 * m.k / ((1.0 + m.nu) * (1.0 + m.nu))
                                  : 2.0 * m.k / ((1.0 - m.nu) * (1.0 - m.nu));
  c.inv2k = 1.0 / (2.0 * m.k);
  c.kappa0 = m.kappa0;
  c.alpha = m.alpha;
  c.beta = m.beta;
  const double en = std::exp(-m.eta);
  c.g_a = (1.0 - m.R) / (1.0 - en);
  c.g_b = (m.R - en) / (1.0 - en);
  c.eta = m.eta;
  c.h = m.h;
  c.c = m.c;
  c.secant = 0;
  c.hterm = m.h_stress ? 1 : 0;
  return c;
}

// ------------------------------------------------------------------ helpers
// B_b^T v for a Voigt vector v (engineering shear), physical derivatives g.
template <int DIM, typename T>
__device__ __forceinline__ void BtV(const T *g, const T *v, T *out) {
  if constexpr (DIM == 1) {
    out[0] = g[0] * v[0];
  } else if constexpr (DIM == 2) {
    out[0] = g[0] * v[0] + g[1] * v[2];
    out[1] = g[1] * v[1] + g[0] * v[2];
  } else {
    out[0] = g[0] * v[0] + g[1] * v[5] + g[2] * v[4];
    out[1] = g[1] * v[1] + g[0] * v[5] + g[2] * v[3];
    out[2] = g[2] * v[2] + g[1] * v[3] + g[0] * v[4];
  }
}

// Isotropic C eps (Voigt, engineering shear).  In 1D lam holds E.
template <int DIM>
__device__ __forceinline__ void iso_stress(double lam, double mu, const double *e, double *s) {
  if constexpr (DIM == 1) {
    s[0] = lam * e[0];
  } else if constexpr (DIM == 2) {
    const double tr = e[0] + e[1];
    s[0] = lam * tr + 2.0 * mu * e[0];
    s[1] = lam * tr + 2.0 * mu * e[1];
    s[2] = mu * e[2];
  } else {
    const double tr = e[0] + e[1] + e[2];
    s[0] = lam * tr + 2.0 * mu * e[0];
    s[1] = lam * tr + 2.0 * mu * e[1];
    s[2] = lam * tr + 2.0 * mu * e[2];
    s[3] = mu * e[3];
    s[4] = mu * e[4];
    s[5] = mu * e[5];
  }
}

// Modified von Mises equivalent strain (Eq. A.3) and its Voigt gradient.
template <int DIM>
__device__ __forceinline__ double equivalent_strain(const MatConst &mc, const double *e, double *d) {
  if constexpr (DIM == 1) {
    d[0] = 1.0;
    return e[0];
  } else {
    constexpr int NV = (DIM == 2) ? 3 : 6;
    double I1, ee;
    if constexpr (DIM == 2) {
      I1 = e[0] + e[1];
      ee = e[0] * e[0] + e[1] * e[1] + 0.5 * e[2] * e[2];
    } else {
      I1 = e[0] + e[1] + e[2];
      ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 0.5 * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
    }
    const double J2 = 0.5 * (ee - I1 * I1 * (1.0 / 3.0));
    const double Q = mc.evm_b2 * I1 * I1 + mc.evm_cJ * J2;
    if (Q > 0.0) {
      const double root = sqrt(Q);
      const double coef = 0.5 * mc.inv2k / root;
      const double nrm = mc.evm_a + coef * 2.0 * mc.evm_b2 * I1;   // common normal part
      const double third = I1 * (1.0 / 3.0);
#pragma unroll
      for (int i = 0; i < DIM; ++i) d[i] = nrm + coef * mc.evm_cJ * (e[i] - third);
#pragma unroll
      for (int i = DIM; i < NV; ++i) d[i] = coef * mc.evm_cJ * 0.5 * e[i];
      return mc.evm_a * I1 + root * mc.inv2k;
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) d[i] = mc.evm_a;
#pragma unroll
    for (int i = DIM; i < NV; ++i) d[i] = 0.0;
    return mc.evm_a * I1;
  }
}

// ------------------------------------------------------------------ element kernel
constexpr int ELEM_THREADS = 128;

template <int ELEM, typename TT, int BT = ELEM_THREADS, bool HT = false>
struct ElemLayout {
  static constexpr int DIM = Elem<ELEM>::DIM, NEN = Elem<ELEM>::NEN, NV = Elem<ELEM>::NV, NVE = Elem<ELEM>::NVE;
  static constexpr bool MIX = Elem<ELEM>::MIXED;
  static constexpr int ND = DIM + 1, NGP = NEN, EPB = BT / NEN;
  static constexpr int DE = MIX ? NVE * DIM : 0;            // micro-strain derivatives (mixed order)
  // double record per Gauss point: dNdx[NEN][DIM], sig dV[NV], rho2, rho4, gbar[DIM] (+ dNe/dx[NVE][DIM])
  static constexpr int RD = NEN * DIM + NV + 2 + DIM + DE;
  static constexpr int O_DN = 0, O_SIG = NEN * DIM, O_R2 = O_SIG + NV, O_R4 = O_R2 + 1, O_GB = O_R4 + 1;
  static constexpr int O_DE = O_GB + DIM;
  // tangent record per Gauss point (TT): dNdx[NEN][DIM], z[NEN][DIM], lam', mu', s[NV], rho1, rho2, rho3,
  // gbar[DIM]; with the h-term stress also q[NEN][DIM] and the coefficients cy, cq of its rank-one terms;
  // with mixed order the micro-strain derivatives dNe/dx[NVE][DIM]
  static constexpr int RT = 2 * NEN * DIM + 2 + NV + 3 + DIM + (HT ? NEN * DIM + 2 : 0) + DE;
  static constexpr int T_DN = 0, T_Z = NEN * DIM, T_LAM = 2 * NEN * DIM, T_MU = T_LAM + 1, T_S = T_MU + 1,
                       T_R1 = T_S + NV, T_R2 = T_R1 + 1, T_R3 = T_R2 + 1, T_GB = T_R3 + 1;
  static constexpr int T_Q = T_GB + DIM, T_CY = T_Q + NEN * DIM, T_CQ = T_CY + 1;
  static constexpr int T_DE = T_GB + DIM + (HT ? NEN * DIM + 2 : 0);
  static constexpr int RDS = (NGP * RD) | 1;                // odd stride: fewer bank conflicts
  static constexpr int RTS = (NGP * RT) | 1;
  static constexpr int SE = MIX ? NGP * NVE * (1 + DIM) : 0;   // micro-strain shape data (mixed order)
  static constexpr size_t BYTES_D = sizeof(double) *
      (size_t)(NGP * NEN + NGP * NEN * DIM + SE + EPB * NEN * DIM + EPB * NEN * ND + EPB * RDS);
  static constexpr size_t bytes(bool res_only) {
    return BYTES_D + (res_only ? 0 : sizeof(TT) * (size_t)(EPB * RTS));
  }
};

// One tile of EPB elements: phase 1 and phase 2 for tile `tile` of an
// element list.  Every thread of the block calls it (it synchronises).
template <int ELEM, typename TT, bool RES_ONLY, int BT = ELEM_THREADS, bool ENERGY = false, bool HT = false>
__device__ __forceinline__ void element_tile(const MeshView &m, const MatConst &mc, const double *__restrict__ u,
                                             const double *__restrict__ kh, const int32_t *__restrict__ elem_list,
                                             int32_t n_elem, TT *__restrict__ Ke, double *__restrict__ re,
                                             int64_t tile, TT *__restrict__ Kcor = nullptr) {
  using L = ElemLayout<ELEM, TT, BT, HT>;
  constexpr int DIM = L::DIM, NEN = L::NEN, NV = L::NV, ND = L::ND, NGP = L::NGP, EPB = L::EPB, NVE = L::NVE;
  constexpr bool MIX = L::MIX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sN = reinterpret_cast<double *>(smem_raw);            // [NGP][NEN]
  double *sdN = sN + NGP * NEN;                                  // [NGP][NEN][DIM]
  double *sNe = sdN + NGP * NEN * DIM;                           // mixed order: [NGP][NVE]
  double *sdNe = sNe + (MIX ? NGP * NVE : 0);                    // mixed order: [NGP][NVE][DIM]
  double *xs = sN + NGP * NEN + NGP * NEN * DIM + L::SE;         // [EPB][NEN][DIM]
  double *us = xs + EPB * NEN * DIM;                             // [EPB][NEN][ND]
  double *recD = us + EPB * NEN * ND;                            // [EPB][RDS]
  TT *recT = reinterpret_cast<TT *>(recD + EPB * L::RDS);        // [EPB][RTS]

  const int tid = threadIdx.x;
  const int el = tid / NEN, a = tid % NEN;
  const int64_t slot = tile * EPB + el;                          // position in the element list
  const bool valid = el < EPB && slot < n_elem;                  // BT need not be a multiple of NEN
  const int32_t e = valid ? (elem_list ? elem_list[slot] : (int32_t)slot) : 0;

  for (int k = tid; k < NGP * NEN; k += BT) sN[k] = shapeU_N<ELEM>(k / NEN, k % NEN);
  for (int k = tid; k < NGP * NEN * DIM; k += BT)
    sdN[k] = shapeU_dN<ELEM>(k / (NEN * DIM), (k / DIM) % NEN, k % DIM);
  if constexpr (MIX) {
    for (int k = tid; k < NGP * NVE; k += BT) sNe[k] = shapeE_N<ELEM>(k / NVE, k % NVE);
    for (int k = tid; k < NGP * NVE * DIM; k += BT)
      sdNe[k] = shapeE_dN<ELEM>(k / (NVE * DIM), (k / DIM) % NVE, k % DIM);
  }
  if (valid) {
    const int32_t node = m.conn[(int64_t)e * NEN + a];
    xs[(el * NEN + a) * DIM + 0] = m.x[node];
    if constexpr (DIM > 1) xs[(el * NEN + a) * DIM + 1] = m.y[node];
    if constexpr (DIM > 2) xs[(el * NEN + a) * DIM + 2] = m.z[node];
#pragma unroll
    for (int i = 0; i < ND; ++i) us[(el * NEN + a) * ND + i] = u[(int64_t)node * ND + i];
  }
  __syncthreads();

  // ---------------- phase 1: Gauss point q = a
  if (valid) {
    const int q = a;
    const double *X = xs + el * NEN * DIM;
    const double *U = us + el * NEN * ND;
    double J[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < NEN; ++b) s += X[b * DIM + i] * sdN[(q * NEN + b) * DIM + j];
        J[i][j] = s;
      }
    double Ji[DIM][DIM], det;
    if constexpr (DIM == 1) {
      det = J[0][0];
      Ji[0][0] = 1.0 / det;
    } else if constexpr (DIM == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double id = 1.0 / det;
      Ji[0][0] = J[1][1] * id;
      Ji[0][1] = -J[0][1] * id;
      Ji[1][0] = -J[1][0] * id;
      Ji[1][1] = J[0][0] * id;
    } else {
      const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      const double id = 1.0 / det;
      Ji[0][0] = c00 * id;
      Ji[1][0] = c01 * id;
      Ji[2][0] = c02 * id;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    }
    double dV = det * m.vol_scale[e];
    if constexpr (MIX) dV *= gp_weight<ELEM>(q);
    // physical derivatives dN_b/dx_i = sum_j dN_b/dxi_j dxi_j/dx_i
    double g[NEN][DIM];
#pragma unroll
    for (int b = 0; b < NEN; ++b)
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) s += sdN[(q * NEN + b) * DIM + j] * Ji[j][i];
        g[b][i] = s;
      }
    // strain eps = sum_b B_b u_b (Voigt, engineering shear)
    double eps[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) eps[v] = 0.0;
    double eb = 0.0, gb[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) gb[i] = 0.0;
#pragma unroll
    for (int b = 0; b < NEN; ++b) {
      const double *ub = U + b * ND;
#pragma unroll
      for (int i = 0; i < DIM; ++i) eps[i] += g[b][i] * ub[i];
      if constexpr (DIM == 2) eps[2] += g[b][1] * ub[0] + g[b][0] * ub[1];
      if constexpr (DIM == 3) {
        eps[3] += g[b][2] * ub[1] + g[b][1] * ub[2];
        eps[4] += g[b][2] * ub[0] + g[b][0] * ub[2];
        eps[5] += g[b][1] * ub[0] + g[b][0] * ub[1];
      }
      if constexpr (!MIX) {
        eb += sN[q * NEN + b] * ub[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) gb[i] += g[b][i] * ub[DIM];
      }
    }
    // mixed order: the micro-equivalent strain lives on the NVE vertex nodes
    double gE[MIX ? NVE : 1][DIM];
    if constexpr (MIX) {
#pragma unroll
      for (int b = 0; b < NVE; ++b) {
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          double s = 0.0;
#pragma unroll
          for (int j = 0; j < DIM; ++j) s += sdNe[(q * NVE + b) * DIM + j] * Ji[j][i];
          gE[b][i] = s;
        }
        const double eb_b = U[b * ND + DIM];
        eb += sNe[q * NVE + b] * eb_b;
#pragma unroll
        for (int i = 0; i < DIM; ++i) gb[i] += gE[b][i] * eb_b;
      }
    }
    double deq[NV];
    const double eq = equivalent_strain<DIM>(mc, eps, deq);
    // trial history (Eq. A.2) and damage (Eq. A.1)
    const double khq = kh[(int64_t)e * NGP + q];
    const bool up = eb > khq;                                    // loading (Eq. A.2)
    const double kap = up ? eb : khq;
    const bool chi = up && !mc.secant;
    double D = 0.0, dD = 0.0;
    if (kap > mc.kappa0) {
      const double ex = exp(-mc.beta * (kap - mc.kappa0));
      const double soft = 1.0 - mc.alpha + mc.alpha * ex;
      const double rk = mc.kappa0 / kap;
      D = 1.0 - rk * soft;
      dD = rk / kap * soft + rk * mc.alpha * mc.beta * ex;
    }
    // interaction (Eq. A.4)
    double gi = 1.0, dgi = -mc.eta * mc.g_a;
    if (D > 0.0) {
      const double en = exp(-mc.eta * D);
      gi = mc.g_a * en + mc.g_b;
      dgi = -mc.eta * mc.g_a * en;
    }
    const double es = m.e_scale[e];
    double ce[NV];
    iso_stress<DIM>(es * mc.lam, es * mc.mu, eps, ce);
    const double omD = 1.0 - D;
    if constexpr (ENERGY) {
      // free energy density (Eq. 1) times dV, one value per Gauss point
      double ece = 0.0, gg = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) ece += eps[v] * ce[v];
#pragma unroll
      for (int i = 0; i < DIM; ++i) gg += gb[i] * gb[i];
      const double de = eq - eb;
      re[slot * NGP + q] = (0.5 * omD * ece + 0.5 * mc.h * de * de + 0.5 * gi * mc.h * mc.c * gg) * dV;
    }
    double *rd = recD + el * L::RDS + q * L::RD;
#pragma unroll
    for (int b = 0; b < NEN; ++b)
#pragma unroll
      for (int i = 0; i < DIM; ++i) rd[L::O_DN + b * DIM + i] = g[b][i];
    const double hdV = mc.h * dV;
#pragma unroll
    for (int v = 0; v < NV; ++v)   // Eq. 2 literal: sigma also carries h (eps_eq - ebar) d eps_eq/d eps
      rd[L::O_SIG + v] = omD * dV * ce[v] + (HT ? hdV * (eq - eb) * deq[v] : 0.0);
    rd[L::O_R2] = gi * mc.h * mc.c * dV;
    rd[L::O_R4] = hdV * (eb - eq);
#pragma unroll
    for (int i = 0; i < DIM; ++i) rd[L::O_GB + i] = gb[i];
    if constexpr (MIX) {
#pragma unroll
      for (int b = 0; b < NVE; ++b)
#pragma unroll
        for (int i = 0; i < DIM; ++i) rd[L::O_DE + b * DIM + i] = gE[b][i];
    }
    if constexpr (!RES_ONLY) {
      TT *rt = recT + el * L::RTS + q * L::RT;
      const double lin = (chi ? dD : 0.0) * dV;      // D' chi dV
      double tv[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) tv[v] = hdV * deq[v];
#pragma unroll
      for (int b = 0; b < NEN; ++b) {
        double z[DIM];
        BtV<DIM, double>(g[b], tv, z);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          rt[L::T_DN + b * DIM + i] = (TT)g[b][i];
          rt[L::T_Z + b * DIM + i] = (TT)z[i];
        }
      }
      rt[L::T_LAM] = (TT)(omD * es * mc.lam * dV);
      rt[L::T_MU] = (TT)(omD * es * mc.mu * dV);
#pragma unroll
      for (int v = 0; v < NV; ++v) rt[L::T_S + v] = (TT)(ce[v] * lin);
      rt[L::T_R1] = (TT)hdV;
      rt[L::T_R2] = (TT)(gi * mc.h * mc.c * dV);
      rt[L::T_R3] = (TT)(mc.h * mc.c * dgi * lin);
#pragma unroll
      for (int i = 0; i < DIM; ++i) rt[L::T_GB + i] = (TT)gb[i];
      if constexpr (MIX) {
#pragma unroll
        for (int b = 0; b < NVE; ++b)
#pragma unroll
          for (int i = 0; i < DIM; ++i) rt[L::T_DE + b * DIM + i] = (TT)gE[b][i];
      }
      if constexpr (HT) {
        // tangent of the h-term stress: h dV [d (x) d + psi d2 eps_eq], psi = eps_eq - ebar.
        // With Q = b2 I1^2 + cJ J2, d2 eps_eq = [d2Q / (2 sqrt Q) - dQ (x) dQ / (4 Q^1.5)] / (2k),
        // d2Q = 2 b2 dI1 (x) dI1 + cJ d2J2, and B_a^T d2J2 B_b = -a_i b_j / 3 + (a_j b_i + a.b delta_ij) / 2:
        // the isotropic parts join lam', mu'; d (x) d and dQ (x) dQ are rank-one (z and q vectors).
        const double hdVp = hdV * (eq - eb);
        double lx = 0.0, mx = 0.0, c3 = 0.0, vq[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) vq[v] = 0.0;
        if constexpr (DIM > 1) {
          double I1 = 0.0, ee = 0.0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) { I1 += eps[i]; ee += eps[i] * eps[i]; }
#pragma unroll
          for (int v = DIM; v < NV; ++v) ee += 0.5 * eps[v] * eps[v];
          const double Q = mc.evm_b2 * I1 * I1 + mc.evm_cJ * 0.5 * (ee - I1 * I1 * (1.0 / 3.0));
          if (Q > 0.0) {
            const double root = sqrt(Q);
            const double c1 = hdVp * mc.inv2k * mc.evm_b2 / root;
            const double c2 = hdVp * mc.inv2k * mc.evm_cJ / (2.0 * root);
            c3 = hdVp * mc.inv2k / (4.0 * Q * root);
            lx = c1 - c2 * (1.0 / 3.0);
            mx = 0.5 * c2;
#pragma unroll
            for (int i = 0; i < DIM; ++i) vq[i] = 2.0 * mc.evm_b2 * I1 + mc.evm_cJ * (eps[i] - I1 * (1.0 / 3.0));
#pragma unroll
            for (int v = DIM; v < NV; ++v) vq[v] = mc.evm_cJ * 0.5 * eps[v];
          }
        }
        rt[L::T_LAM] = (TT)(omD * es * mc.lam * dV + lx);
        rt[L::T_MU] = (TT)(omD * es * mc.mu * dV + mx);
#pragma unroll
        for (int b = 0; b < NEN; ++b) {
          double qb[DIM];
          BtV<DIM, double>(g[b], vq, qb);
#pragma unroll
          for (int i = 0; i < DIM; ++i) rt[L::T_Q + b * DIM + i] = (TT)qb[i];
        }
        rt[L::T_CY] = (TT)(hdV > 0.0 ? 1.0 / hdV : 0.0);   // h dV (B^T d)(B^T d)^T = z z^T / (h dV)
        rt[L::T_CQ] = (TT)(-c3);
      }
    }
  }
  __syncthreads();
  if (!valid) return;                                            // no barrier follows in this tile
  if constexpr (ENERGY) return;

  // ---------------- phase 2: block row a
  const double *RD0 = recD + el * L::RDS;
  {
    double ru[DIM], rep = 0.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) ru[i] = 0.0;
#pragma unroll
    for (int q = 0; q < NGP; ++q) {
      const double *rd = RD0 + q * L::RD;
      const double *A = rd + L::O_DN + a * DIM;
      double t[DIM];
      BtV<DIM, double>(A, rd + L::O_SIG, t);
#pragma unroll
      for (int i = 0; i < DIM; ++i) ru[i] += t[i];
      if constexpr (!MIX) {
        double ag = 0.0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) ag += A[i] * rd[L::O_GB + i];
        rep += sN[q * NEN + a] * rd[L::O_R4] + rd[L::O_R2] * ag;
      } else if (a < NVE) {                        // micro-strain rows: vertex nodes only
        const double *Ae = rd + L::O_DE + a * DIM;
        double ag = 0.0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) ag += Ae[i] * rd[L::O_GB + i];
        rep += sNe[q * NVE + a] * rd[L::O_R4] + rd[L::O_R2] * ag;
      }
    }
    double *rout = re + ((int64_t)slot * NEN + a) * ND;
#pragma unroll
    for (int i = 0; i < DIM; ++i) rout[i] = ru[i];
    rout[DIM] = rep;
  }
  if constexpr (!RES_ONLY) {
    const TT *RT0 = recT + el * L::RTS;
    constexpr int BC = (NEN <= 4) ? NEN : (NEN % 4 == 0) ? 4 : 3;   // b columns per pass (register budget)
    // mixed order: the micro-strain shape data of row node a (zero off the vertices)
    const bool aE = !MIX || a < NVE;
    const int ai = aE ? a : 0;
#pragma unroll 1
    for (int b0 = 0; b0 < NEN; b0 += BC) {
      TT acc[ND][BC][ND];
#pragma unroll
      for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int bb = 0; bb < BC; ++bb)
#pragma unroll
          for (int j = 0; j < ND; ++j) acc[i][bb][j] = (TT)0;
#pragma unroll
      for (int q = 0; q < NGP; ++q) {
        const TT *rt = RT0 + q * L::RT;
        TT A[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) A[i] = rt[L::T_DN + a * DIM + i];
        const TT lamp = rt[L::T_LAM], mup = rt[L::T_MU];
        TT Na, Ae[DIM];
        if constexpr (!MIX) {
          Na = (TT)sN[q * NEN + a];
#pragma unroll
          for (int i = 0; i < DIM; ++i) Ae[i] = A[i];
        } else {
          Na = aE ? (TT)sNe[q * NVE + ai] : (TT)0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) Ae[i] = aE ? rt[L::T_DE + ai * DIM + i] : (TT)0;
        }
        TT la[DIM], ma[DIM], l2m[DIM], w[DIM], fa[DIM];
        TT ag = (TT)0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          la[i] = lamp * A[i];
          ma[i] = mup * A[i];
          l2m[i] = la[i] + (TT)2 * ma[i];
          fa[i] = rt[L::T_R2] * Ae[i];
          ag += Ae[i] * rt[L::T_GB + i];
        }
        BtV<DIM, TT>(A, rt + L::T_S, w);               // B_a^T (C eps) D' chi dV
        const TT ea = Na * rt[L::T_R1] + rt[L::T_R3] * ag;
        const TT nNa = -Na;
        TT cza[DIM], cqa[DIM];                         // h-term stress: rank-one factors of row node a
        if constexpr (HT) {
          const TT cy = rt[L::T_CY], cq = rt[L::T_CQ];
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            const TT za = rt[L::T_Z + a * DIM + i];
            w[i] += za;                                // K_ue gains -B_a^T h d N_b dV
            cza[i] = cy * za;
            cqa[i] = cq * rt[L::T_Q + a * DIM + i];
          }
        }
#pragma unroll
        for (int bb = 0; bb < BC; ++bb) {
          const int b = b0 + bb;
          const TT *B = rt + L::T_DN + b * DIM;
          const TT *Z = rt + L::T_Z + b * DIM;
          TT Nb, Bv[DIM], BvE[DIM];
#pragma unroll
          for (int k = 0; k < DIM; ++k) Bv[k] = B[k];
          if constexpr (!MIX) {
            Nb = (TT)shape_N<DIM>(q, b);
#pragma unroll
            for (int k = 0; k < DIM; ++k) BvE[k] = Bv[k];
          } else {
            const bool bE = b < NVE;
            const int bi = bE ? b : 0;
            Nb = bE ? (TT)sNe[q * NVE + bi] : (TT)0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) BvE[k] = bE ? rt[L::T_DE + bi * DIM + k] : (TT)0;
          }
          // K_uu (Eq. 11a): lam' a_i b_j + mu' a_j b_i + mu' (a.b) delta_ij
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
              if (i == j) {
                TT s = acc[i][bb][i] + l2m[i] * Bv[i];
#pragma unroll
                for (int k = 0; k < DIM; ++k)
                  if (k != i) s += ma[k] * Bv[k];
                acc[i][bb][i] = s;
              } else {
                acc[i][bb][j] += la[i] * Bv[j] + ma[j] * Bv[i];
              }
            }
          if constexpr (HT) {
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) acc[i][bb][j] += cza[i] * Z[j] + cqa[i] * rt[L::T_Q + b * DIM + j];
          }
          // K_ue (Eq. 11b) and K_eu (Eq. 11c)
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            acc[i][bb][DIM] -= w[i] * Nb;
            acc[DIM][bb][i] += nNa * Z[i];
          }
          // K_ee (Eq. 11d)
          TT s = acc[DIM][bb][DIM] + ea * Nb;
#pragma unroll
          for (int k = 0; k < DIM; ++k) s += fa[k] * BvE[k];
          acc[DIM][bb][DIM] = s;
        }
      }
      TT *kout = Ke + ((int64_t)slot * NEN + a) * ND * (NEN * ND) + b0 * ND;
#pragma unroll
      for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int bb = 0; bb < BC; ++bb)
#pragma unroll
          for (int j = 0; j < ND; ++j) kout[i * NEN * ND + bb * ND + j] = acc[i][bb][j];
    }
    if (Kcor) {
      // the loading-indicator terms of the block row (the D'(kappa) chi terms
      // of Eq. 11b and 11d, included above): the secant tangent is the
      // consistent one minus them.  They sit in the micro-strain column of
      // every node block: nd values per column node b.
      TT cor[NEN][ND];
#pragma unroll
      for (int b = 0; b < NEN; ++b)
#pragma unroll
        for (int i = 0; i < ND; ++i) cor[b][i] = (TT)0;
#pragma unroll
      for (int q = 0; q < NGP; ++q) {
        const TT *rt = RT0 + q * L::RT;
        TT A[DIM], w[DIM];
        TT ag = (TT)0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          A[i] = rt[L::T_DN + a * DIM + i];
          const TT Ae = MIX ? (aE ? rt[L::T_DE + ai * DIM + i] : (TT)0) : A[i];
          ag += Ae * rt[L::T_GB + i];
        }
        BtV<DIM, TT>(A, rt + L::T_S, w);
        const TT er = rt[L::T_R3] * ag;
#pragma unroll
        for (int b = 0; b < NEN; ++b) {
          TT Nb;
          if constexpr (!MIX) Nb = (TT)shape_N<DIM>(q, b);
          else Nb = (b < NVE) ? (TT)sNe[q * NVE + (b < NVE ? b : 0)] : (TT)0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) cor[b][i] -= w[i] * Nb;
          cor[b][DIM] += er * Nb;
        }
      }
      TT *cout_ = Kcor + ((int64_t)slot * NEN + a) * NEN * ND;
#pragma unroll
      for (int b = 0; b < NEN; ++b)
#pragma unroll
        for (int i = 0; i < ND; ++i) cout_[b * ND + i] = cor[b][i];
    }
  }
}

template <int ELEM, typename TT, bool RES_ONLY, bool HT>
__global__ void __launch_bounds__(ELEM_THREADS)
element_kernel(MeshView m, MatConst mc, const double *__restrict__ u, const double *__restrict__ kh,
               const int32_t *__restrict__ elem_list, int32_t n_elem, TT *__restrict__ Ke,
               double *__restrict__ re) {
  element_tile<ELEM, TT, RES_ONLY, ELEM_THREADS, false, HT>(m, mc, u, kh, elem_list, n_elem, Ke, re, blockIdx.x);
}

template <int ELEM, typename TT, bool RES_ONLY, bool HT>
static cudaError_t launch_element_t(const MeshView &m, const MatConst &mc, const double *u,
                                    const double *kh, const int32_t *list, int32_t n, TT *Ke, double *re,
                                    cudaStream_t s) {
  using L = ElemLayout<ELEM, TT, ELEM_THREADS, HT>;
  if (n <= 0) return cudaSuccess;
  const size_t smem = L::bytes(RES_ONLY);
  auto fn = element_kernel<ELEM, TT, RES_ONLY, HT>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int grid = (n + L::EPB - 1) / L::EPB;
  fn<<<grid, ELEM_THREADS, smem, s>>>(m, mc, u, kh, list, n, Ke, re);
  return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_element(int elem, const MeshView &m, const MatConst &mc, const double *u,
                           const double *kh, const int32_t *list, int32_t n, TT *Ke, double *re,
                           bool res_only, cudaStream_t s) {
#define LGDM_EL(E)                                                                                          \
  if (mc.hterm)                                                                                             \
    return res_only ? launch_element_t<E, TT, true, true>(m, mc, u, kh, list, n, Ke, re, s)                 \
                    : launch_element_t<E, TT, false, true>(m, mc, u, kh, list, n, Ke, re, s);               \
  return res_only ? launch_element_t<E, TT, true, false>(m, mc, u, kh, list, n, Ke, re, s)                  \
                  : launch_element_t<E, TT, false, false>(m, mc, u, kh, list, n, Ke, re, s)
  switch (elem) {
    case LGDM_L2: LGDM_EL(LGDM_L2);
    case LGDM_Q4: LGDM_EL(LGDM_Q4);
    case LGDM_H8: LGDM_EL(LGDM_H8);
    case LGDM_L3: LGDM_EL(LGDM_L3);
    case LGDM_Q9: LGDM_EL(LGDM_Q9);
  }
#undef LGDM_EL
  return cudaErrorInvalidValue;
}
template cudaError_t launch_element<double>(int, const MeshView &, const MatConst &, const double *,
                                            const double *, const int32_t *, int32_t, double *,
                                            double *, bool, cudaStream_t);
template cudaError_t launch_element<float>(int, const MeshView &, const MatConst &, const double *,
                                           const double *, const int32_t *, int32_t, float *, double *,
                                           bool, cudaStream_t);

// ------------------------------------------------------------------ gather
template <int ND, int NEN, typename TT>
__device__ __forceinline__ void gather_pair(const PatternView &p, const TT *__restrict__ Ke,
                                            const double *__restrict__ re, TT *__restrict__ vals,
                                            double *__restrict__ rraw, double *__restrict__ rhs, int64_t pr,
                                            const TT *__restrict__ Kcor = nullptr, TT *__restrict__ vsec = nullptr) {
  if (pr >= p.npairs) return;
  const int32_t a = p.pair_node[pr], b = p.nbr[pr];
  const int32_t pb = p.nbr_ptr[a];
  const int32_t deg = p.nbr_ptr[a + 1] - pb;
  const int32_t s = (int32_t)(pr - pb);
  const bool diag = (a == b);
  TT acc[ND][ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) acc[i][j] = (TT)0;
  double racc[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) racc[i] = 0.0;
  TT cacc[ND];                                   // loading-indicator terms (secant = consistent - them)
#pragma unroll
  for (int i = 0; i < ND; ++i) cacc[i] = (TT)0;
  constexpr int LB = (NEN > 8) ? 4 : 3;          // bits per local node in the packed contribution
  const int32_t c1 = p.pc_ptr[pr + 1];
  for (int32_t c = p.pc_ptr[pr]; c < c1; ++c) {
    const int32_t pk = p.pc[c];
    const int64_t e = pk >> (2 * LB);
    const int al = (pk >> LB) & ((1 << LB) - 1), bl = pk & ((1 << LB) - 1);
    const TT *blk = Ke + ((e * NEN + al) * ND) * (NEN * ND) + bl * ND;
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
      for (int j = 0; j < ND; ++j) acc[i][j] += blk[i * NEN * ND + j];
    if (vsec) {
      const TT *cb = Kcor + ((e * NEN + al) * NEN + bl) * ND;
#pragma unroll
      for (int i = 0; i < ND; ++i) cacc[i] += cb[i];
    }
    if (diag) {
      const double *rb = re + (e * NEN + al) * ND;
#pragma unroll
      for (int i = 0; i < ND; ++i) racc[i] += rb[i];
    }
  }
  const int64_t vbase = (int64_t)ND * ND * pb + (int64_t)ND * s;
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    const int64_t row = (int64_t)ND * a + i;
    const bool rdir = p.isdir[row];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int64_t col = (int64_t)ND * b + j;
      const bool dir = rdir || p.isdir[col];
      TT v = acc[i][j];
      if (dir) v = (row == col) ? (TT)1 : (TT)0;
      vals[vbase + (int64_t)i * ND * deg + j] = v;
      if (vsec) vsec[vbase + (int64_t)i * ND * deg + j] = dir ? v : (j == ND - 1 ? acc[i][j] - cacc[i] : acc[i][j]);
    }
    if (diag) {
      rraw[row] = racc[i];
      rhs[row] = rdir ? 0.0 : -racc[i];
    }
  }
}

template <int ND, int NEN, typename TT>
__global__ void __launch_bounds__(256)
gather_kernel(PatternView p, const TT *__restrict__ Ke, const double *__restrict__ re,
              TT *__restrict__ vals, double *__restrict__ rraw, double *__restrict__ rhs) {
  gather_pair<ND, NEN, TT>(p, Ke, re, vals, rraw, rhs, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename TT>
cudaError_t launch_gather(int elem, const PatternView &p, const TT *Ke, const double *re, TT *vals,
                          double *rraw, double *rhs, cudaStream_t s) {
  const int grid = (int)((p.npairs + 255) / 256);
  switch (elem) {
    case LGDM_L2: gather_kernel<2, 2, TT><<<grid, 256, 0, s>>>(p, Ke, re, vals, rraw, rhs); break;
    case LGDM_Q4: gather_kernel<3, 4, TT><<<grid, 256, 0, s>>>(p, Ke, re, vals, rraw, rhs); break;
    case LGDM_H8: gather_kernel<4, 8, TT><<<grid, 256, 0, s>>>(p, Ke, re, vals, rraw, rhs); break;
    case LGDM_L3: gather_kernel<2, 3, TT><<<grid, 256, 0, s>>>(p, Ke, re, vals, rraw, rhs); break;
    case LGDM_Q9: gather_kernel<3, 9, TT><<<grid, 256, 0, s>>>(p, Ke, re, vals, rraw, rhs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_gather<double>(int, const PatternView &, const double *, const double *,
                                           double *, double *, double *, cudaStream_t);
template cudaError_t launch_gather<float>(int, const PatternView &, const float *, const double *,
                                          float *, double *, double *, cudaStream_t);

// ------------------------------------------------------------------ preconditioner
template <int ND, typename TT>
__global__ void precond_kernel(PatternView p, const TT *__restrict__ vals, int kind, TT *__restrict__ minv) {
  precond_node<ND, TT>(p, vals, kind, minv, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename TT>
cudaError_t launch_precond(int nd, const PatternView &p, const TT *vals, int kind, TT *minv, cudaStream_t s) {
  const int grid = (p.nnode + 127) / 128;
  switch (nd) {
    case 2: precond_kernel<2, TT><<<grid, 128, 0, s>>>(p, vals, kind, minv); break;
    case 3: precond_kernel<3, TT><<<grid, 128, 0, s>>>(p, vals, kind, minv); break;
    case 4: precond_kernel<4, TT><<<grid, 128, 0, s>>>(p, vals, kind, minv); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_precond<double>(int, const PatternView &, const double *, int, double *, cudaStream_t);
template cudaError_t launch_precond<float>(int, const PatternView &, const float *, int, float *, cudaStream_t);

// ------------------------------------------------------------------ small kernels
__global__ void set_dirichlet_kernel(double *u, const int32_t *dof, const double *scale, int32_t n, double load) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[dof[i]] = scale[i] * load;
}
cudaError_t launch_set_dirichlet(double *u, const int32_t *dof, const double *scale, int32_t n, double load,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  set_dirichlet_kernel<<<(n + 255) / 256, 256, 0, s>>>(u, dof, scale, n, load);
  return cudaGetLastError();
}

int elem_nen(int elem) {
  switch (elem) {
    case LGDM_L2: return 2;
    case LGDM_Q4: return 4;
    case LGDM_H8: return 8;
    case LGDM_L3: return 3;
    case LGDM_Q9: return 9;
  }
  return 0;
}

// History commit (Eq. A.2): kappa_hist <- max(kappa_hist, ebar at the Gauss point).
template <int ELEM>
__global__ void commit_kernel(MeshView m, const double *__restrict__ u, double *__restrict__ kh) {
  constexpr int DIM = Elem<ELEM>::DIM, NEN = Elem<ELEM>::NEN, NVE = Elem<ELEM>::NVE, ND = DIM + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m.nel * NEN) return;
  const int64_t e = t / NEN;
  const int q = (int)(t % NEN);
  double eb = 0.0;
#pragma unroll
  for (int b = 0; b < NVE; ++b) eb += shapeE_N<ELEM>(q, b) * u[(int64_t)m.conn[e * NEN + b] * ND + DIM];
  kh[t] = fmax(kh[t], eb);
}
cudaError_t launch_commit(int elem, const MeshView &m, const double *u, double *kh, cudaStream_t s) {
  const int nen = elem_nen(elem);
  const int64_t n = (int64_t)m.nel * nen;
  const int grid = (int)((n + 255) / 256);
  switch (elem) {
    case LGDM_L2: commit_kernel<LGDM_L2><<<grid, 256, 0, s>>>(m, u, kh); break;
    case LGDM_Q4: commit_kernel<LGDM_Q4><<<grid, 256, 0, s>>>(m, u, kh); break;
    case LGDM_H8: commit_kernel<LGDM_H8><<<grid, 256, 0, s>>>(m, u, kh); break;
    case LGDM_L3: commit_kernel<LGDM_L3><<<grid, 256, 0, s>>>(m, u, kh); break;
    case LGDM_Q9: commit_kernel<LGDM_Q9><<<grid, 256, 0, s>>>(m, u, kh); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void fill_kernel(double *p, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
cudaError_t launch_fill(double *p, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

__global__ void diag_pairs_kernel(PatternView p, int32_t *diag) {
  const int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= p.nnode) return;
  int32_t k = p.nbr_ptr[a];
  const int32_t k1 = p.nbr_ptr[a + 1];
  while (k < k1 && p.nbr[k] != a) ++k;
  diag[a] = (k < k1) ? k : p.nbr_ptr[a];
}
cudaError_t launch_diag_pairs(const PatternView &p, int32_t *diag, cudaStream_t s) {
  diag_pairs_kernel<<<(p.nnode + 255) / 256, 256, 0, s>>>(p, diag);
  return cudaGetLastError();
}

template <int ELEM>
__global__ void __launch_bounds__(ELEM_THREADS)
energy_kernel(MeshView m, MatConst mc, const double *__restrict__ u, const double *__restrict__ kh,
              int32_t n_elem, double *__restrict__ psi) {
  element_tile<ELEM, double, true, ELEM_THREADS, true>(m, mc, u, kh, nullptr, n_elem, nullptr, psi, blockIdx.x);
}

// Sum of n values in a fixed order: 256-thread blocks sum fixed chunks in a
// fixed tree, one block adds the block sums in order.
__global__ void chunk_sum_kernel(const double *__restrict__ x, int64_t n, int64_t chunk, double *__restrict__ part) {
  __shared__ double sh[256];
  const int64_t lo = blockIdx.x * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += 256) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

cudaError_t launch_energy(int elem, const MeshView &m, const MatConst &mc, const double *u, const double *kh,
                          double *psi, double *part, double *out, cudaStream_t s) {
  const int nen = elem_nen(elem);
  const int epb = ELEM_THREADS / nen;
  const int grid = (m.nel + epb - 1) / epb;
  size_t smem = 0;
  cudaError_t err = cudaSuccess;
#define LGDM_EN(E)                                                                                   \
  smem = ElemLayout<E, double>::bytes(true);                                                         \
  err = cudaFuncSetAttribute(energy_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  if (err != cudaSuccess) return err;                                                                \
  energy_kernel<E><<<grid, ELEM_THREADS, smem, s>>>(m, mc, u, kh, m.nel, psi);                       \
  break
  switch (elem) {
    case LGDM_L2: LGDM_EN(LGDM_L2);
    case LGDM_Q4: LGDM_EN(LGDM_Q4);
    case LGDM_H8: LGDM_EN(LGDM_H8);
    case LGDM_L3: LGDM_EN(LGDM_L3);
    case LGDM_Q9: LGDM_EN(LGDM_Q9);
    default: return cudaErrorInvalidValue;
  }
#undef LGDM_EN
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t n = (int64_t)m.nel * nen;
  const int64_t chunk = 4096;
  const int nblk = (int)((n + chunk - 1) / chunk);
  chunk_sum_kernel<<<nblk, 256, 0, s>>>(psi, n, chunk, part);
  chunk_sum_kernel<<<1, 256, 0, s>>>(part, nblk, nblk, out);
  return cudaGetLastError();
}

__global__ void damage_field_kernel(MatConst mc, const double *kh, int64_t n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double k = kh[i];
  double D = 0.0;
  if (k > mc.kappa0) D = 1.0 - mc.kappa0 / k * (1.0 - mc.alpha + mc.alpha * exp(-mc.beta * (k - mc.kappa0)));
  out[i] = D;
}
cudaError_t launch_damage_field(const MatConst &mc, const double *kh, int64_t n, double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  damage_field_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(mc, kh, n, out);
  return cudaGetLastError();
}

// Reaction: sum_k w[k] re[idx[k]], one block, fixed summation order.
__global__ void reaction_sum_kernel(const double *re, const int32_t *idx, const double *w, int32_t n, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int32_t k = threadIdx.x; k < n; k += 256) s += w[k] * re[idx[k]];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
cudaError_t launch_reaction_sum(const double *re, const int32_t *idx, const double *w, int32_t n, double *out,
                                cudaStream_t s) {
  reaction_sum_kernel<<<1, 256, 0, s>>>(re, idx, w, n, out);
  return cudaGetLastError();
}

__global__ void external_work_kernel(double *c, double dload) {
  c[1] += 0.5 * (c[0] + c[2]) * dload;
  c[2] = c[0];
}
cudaError_t launch_external_work(double *c, double dload, cudaStream_t s) {
  external_work_kernel<<<1, 1, 0, s>>>(c, dload);
  return cudaGetLastError();
}

// w_q det J at Gauss point q of element e.
template <int ELEM>
__device__ __forceinline__ double gp_det(const MeshView &m, int64_t e, int q) {
  constexpr int DIM = Elem<ELEM>::DIM, NEN = Elem<ELEM>::NEN;
  double J[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) J[i][j] = 0.0;
#pragma unroll
  for (int b = 0; b < NEN; ++b) {
    const int32_t node = m.conn[e * NEN + b];
    const double X[3] = {m.x[node], DIM > 1 ? m.y[node] : 0.0, DIM > 2 ? m.z[node] : 0.0};
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) J[i][j] += X[i] * shapeU_dN<ELEM>(q, b, j);
  }
  double det;
  if constexpr (DIM == 1) det = J[0][0];
  else if constexpr (DIM == 2) det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  else
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) + J[0][1] * (J[1][2] * J[2][0] - J[1][0] * J[2][2]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if constexpr (Elem<ELEM>::MIXED) det *= gp_weight<ELEM>(q);
  return det;
}

template <int ELEM>
__global__ void damaged_volume_kernel(MeshView m, MatConst mc, const double *__restrict__ kh, double thr,
                                      double *__restrict__ vol) {
  constexpr int NEN = Elem<ELEM>::NEN;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m.nel * NEN) return;
  const int64_t e = t / NEN;
  const double k = kh[t];
  double D = 0.0;
  if (k > mc.kappa0) D = 1.0 - mc.kappa0 / k * (1.0 - mc.alpha + mc.alpha * exp(-mc.beta * (k - mc.kappa0)));
  vol[t] = (D > thr) ? gp_det<ELEM>(m, e, (int)(t % NEN)) * m.vol_scale[e] : 0.0;
}

cudaError_t launch_damaged_volume(int elem, const MeshView &m, const MatConst &mc, const double *kh, double thr,
                                  double *vol, double *part, double *out, cudaStream_t s) {
  const int nen = elem_nen(elem);
  const int64_t n = (int64_t)m.nel * nen;
  const int grid = (int)((n + 255) / 256);
  switch (elem) {
    case LGDM_L2: damaged_volume_kernel<LGDM_L2><<<grid, 256, 0, s>>>(m, mc, kh, thr, vol); break;
    case LGDM_Q4: damaged_volume_kernel<LGDM_Q4><<<grid, 256, 0, s>>>(m, mc, kh, thr, vol); break;
    case LGDM_H8: damaged_volume_kernel<LGDM_H8><<<grid, 256, 0, s>>>(m, mc, kh, thr, vol); break;
    case LGDM_L3: damaged_volume_kernel<LGDM_L3><<<grid, 256, 0, s>>>(m, mc, kh, thr, vol); break;
    case LGDM_Q9: damaged_volume_kernel<LGDM_Q9><<<grid, 256, 0, s>>>(m, mc, kh, thr, vol); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t chunk = 4096;
  const int nblk = (int)((n + chunk - 1) / chunk);
  chunk_sum_kernel<<<nblk, 256, 0, s>>>(vol, n, chunk, part);
  chunk_sum_kernel<<<1, 256, 0, s>>>(part, nblk, nblk, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ batched kernels
// Persistent: a grid of a few blocks per SM walks all members' tiles.
template <int ELEM, typename TT, int BT, bool HT>
__global__ void __launch_bounds__(BT)
batch_element_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                     const int64_t *__restrict__ tile_start, int nm, int64_t total, const int32_t *__restrict__ active) {
  for (int64_t k = blockIdx.x; k < total; k += gridDim.x) {
    const int j = find_member(tile_start, nm, k);
    const int sm = members[j];
    if (active[sm]) {
      const BatchSim &d = sims[sm];
      element_tile<ELEM, TT, false, BT, false, HT>(d.m, d.mc, d.u, d.kh, nullptr, d.m.nel, static_cast<TT *>(d.Ke),
                                                   d.re, k - tile_start[j], static_cast<TT *>(d.Kcor));
    }
    __syncthreads();
  }
}

template <int ND, int NEN, typename TT>
__global__ void __launch_bounds__(256)
batch_gather_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                    const int64_t *__restrict__ block_start, int nm, const int32_t *__restrict__ active) {
  const int j = find_member(block_start, nm, blockIdx.x);
  const int sm = members[j];
  if (!active[sm]) return;
  const BatchSim &d = sims[sm];
  gather_pair<ND, NEN, TT>(d.p, static_cast<const TT *>(d.Ke), d.re, static_cast<TT *>(d.vals), d.rraw, d.rhs,
                           (blockIdx.x - block_start[j]) * 256 + threadIdx.x, static_cast<const TT *>(d.Kcor),
                           static_cast<TT *>(d.vals_sec));
}

template <int ND, typename TT>
__global__ void __launch_bounds__(128)
batch_precond_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                     const int64_t *__restrict__ block_start, int nm, const int32_t *__restrict__ active) {
  const int j = find_member(block_start, nm, blockIdx.x);
  const int sm = members[j];
  if (!active[sm]) return;
  const BatchSim &d = sims[sm];
  // with the multigrid, the smoother of the system level is built from the secant matrix
  precond_node<ND, TT>(d.p, static_cast<const TT *>(d.vals_sec ? d.vals_sec : d.vals), d.precond,
                       static_cast<TT *>(d.minv),
                       (int32_t)((blockIdx.x - block_start[j]) * 128 + threadIdx.x));
}

template <int ELEM, typename TT, int BT, bool HT>
static cudaError_t launch_batch_element_t(const BatchSim *sims, const int32_t *members, const int64_t *tile_start,
                                          int nm, int64_t total, const int32_t *active, int grid, cudaStream_t s) {
  using L = ElemLayout<ELEM, TT, BT, HT>;
  const size_t smem = L::bytes(false);
  auto fn = batch_element_kernel<ELEM, TT, BT, HT>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  fn<<<grid, BT, smem, s>>>(sims, members, tile_start, nm, total, active);
  return cudaGetLastError();
}

// Largest element block size <= bt (256, 128, 64) whose shared-memory layout
// fits the 227 KB a block may opt in to (the FP64 8-node and 9-node layouts
// with the h-term stress do not fit at 256 threads).
constexpr size_t SMEM_OPTIN = 232448;
template <int E, typename TT, bool H>
int fit_block(int bt) {
  while (bt > 64) {
    const size_t b = (bt >= 256) ? ElemLayout<E, TT, 256, H>::bytes(false) : ElemLayout<E, TT, 128, H>::bytes(false);
    if (b <= SMEM_OPTIN) return bt;
    bt /= 2;
  }
  return 64;
}
template <typename TT, bool H>
int fit_block_e(int elem, int bt) {
  switch (elem) {
    case LGDM_L2: return fit_block<LGDM_L2, TT, H>(bt);
    case LGDM_Q4: return fit_block<LGDM_Q4, TT, H>(bt);
    case LGDM_H8: return fit_block<LGDM_H8, TT, H>(bt);
    case LGDM_L3: return fit_block<LGDM_L3, TT, H>(bt);
    case LGDM_Q9: return fit_block<LGDM_Q9, TT, H>(bt);
  }
  return bt;
}
int element_block(int elem, bool fp32, bool hterm, int bt) {
  if (fp32) return hterm ? fit_block_e<float, true>(elem, bt) : fit_block_e<float, false>(elem, bt);
  return hterm ? fit_block_e<double, true>(elem, bt) : fit_block_e<double, false>(elem, bt);
}

int batch_tile_elements(int elem, bool fp32, bool hterm, int bt) {
  return element_block(elem, fp32, hterm, bt) / elem_nen(elem);
}

template <typename TT>
cudaError_t launch_batch_element(int elem, int bt, bool hterm, const BatchSim *sims, const int32_t *members,
                                 const int64_t *tile_start, int nm, int64_t total, const int32_t *active, int grid,
                                 cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  bt = element_block(elem, sizeof(TT) == 4, hterm, bt);
#define LGDM_BE2(E, H)                                                                                            \
  switch (bt) {                                                                                                   \
    case 64: return launch_batch_element_t<E, TT, 64, H>(sims, members, tile_start, nm, total, active, grid, s);   \
    case 128: return launch_batch_element_t<E, TT, 128, H>(sims, members, tile_start, nm, total, active, grid, s); \
    case 256: return launch_batch_element_t<E, TT, 256, H>(sims, members, tile_start, nm, total, active, grid, s); \
  }                                                                                                               \
  return cudaErrorInvalidValue
#define LGDM_BE(E)          \
  if (hterm) {              \
    LGDM_BE2(E, true);      \
  } else {                  \
    LGDM_BE2(E, false);     \
  }
  switch (elem) {
    case LGDM_L2: LGDM_BE(LGDM_L2);
    case LGDM_Q4: LGDM_BE(LGDM_Q4);
    case LGDM_H8: LGDM_BE(LGDM_H8);
    case LGDM_L3: LGDM_BE(LGDM_L3);
    case LGDM_Q9: LGDM_BE(LGDM_Q9);
  }
#undef LGDM_BE
#undef LGDM_BE2
  return cudaErrorInvalidValue;
}
template cudaError_t launch_batch_element<double>(int, int, bool, const BatchSim *, const int32_t *, const int64_t *,
                                                  int, int64_t, const int32_t *, int, cudaStream_t);
template cudaError_t launch_batch_element<float>(int, int, bool, const BatchSim *, const int32_t *, const int64_t *,
                                                 int, int64_t, const int32_t *, int, cudaStream_t);

template <typename TT>
cudaError_t launch_batch_gather(int elem, const BatchSim *sims, const int32_t *members, const int64_t *block_start,
                                int nm, int64_t total_blocks, const int32_t *active, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  switch (elem) {
    case LGDM_L2: batch_gather_kernel<2, 2, TT><<<(unsigned)total_blocks, 256, 0, s>>>(sims, members, block_start, nm, active); break;
    case LGDM_Q4: batch_gather_kernel<3, 4, TT><<<(unsigned)total_blocks, 256, 0, s>>>(sims, members, block_start, nm, active); break;
    case LGDM_H8: batch_gather_kernel<4, 8, TT><<<(unsigned)total_blocks, 256, 0, s>>>(sims, members, block_start, nm, active); break;
    case LGDM_L3: batch_gather_kernel<2, 3, TT><<<(unsigned)total_blocks, 256, 0, s>>>(sims, members, block_start, nm, active); break;
    case LGDM_Q9: batch_gather_kernel<3, 9, TT><<<(unsigned)total_blocks, 256, 0, s>>>(sims, members, block_start, nm, active); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_batch_gather<double>(int, const BatchSim *, const int32_t *, const int64_t *, int, int64_t,
                                                 const int32_t *, cudaStream_t);
template cudaError_t launch_batch_gather<float>(int, const BatchSim *, const int32_t *, const int64_t *, int, int64_t,
                                                const int32_t *, cudaStream_t);

template <typename TT>
cudaError_t launch_batch_precond(int nd, const BatchSim *sims, const int32_t *members, const int64_t *block_start,
                                 int nm, int64_t total_blocks, const int32_t *active, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  switch (nd) {
    case 2: batch_precond_kernel<2, TT><<<(unsigned)total_blocks, 128, 0, s>>>(sims, members, block_start, nm, active); break;
    case 3: batch_precond_kernel<3, TT><<<(unsigned)total_blocks, 128, 0, s>>>(sims, members, block_start, nm, active); break;
    case 4: batch_precond_kernel<4, TT><<<(unsigned)total_blocks, 128, 0, s>>>(sims, members, block_start, nm, active); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_batch_precond<double>(int, const BatchSim *, const int32_t *, const int64_t *, int, int64_t,
                                                  const int32_t *, cudaStream_t);
template cudaError_t launch_batch_precond<float>(int, const BatchSim *, const int32_t *, const int64_t *, int, int64_t,
                                                 const int32_t *, cudaStream_t);

}  // namespace lgdm
