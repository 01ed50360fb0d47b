/*
 * CPU FP64 oracle of the two-fluid spin-SPH time step.  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add), OpenMP over the
 * rows i only; every j loop runs j = 0..n-1 in ascending order.
 *
 * Model followed (Sec. 2.1, Eqs. 1, 2 and 4; Algorithm 1; Sec. 3 set-up):
 *   M0  Wendland C2 kernel, support 2h; F = -(1/r) dW/dr >= 0.
 *   M1  rho_i = sum_j m_j W_ij (self included) for fluid and inner walls;
 *       outer walls keep rho0 (wall and dummy particles, Sec. 3).
 *   M2  Tait equation of state, Eq. 4.
 *   M3  symmetric pressure gradient  m_i m_j (P_i/rho_i^2 + P_j/rho_j^2) F r_ij.
 *   M4  interfacial force C_T V_i V_j F P_h r_ij between unlike species: the
 *       +/- rho_s sigma grad T pair of Eqs. 1-2 with equal particle volumes,
 *       acting in the horizontal plane only (Sec. 2.1).
 *   M5  central shear viscosity  -10 (eta - 0.6 eta_r) V_i V_j F (e.v_ij) e.
 *   M6  transverse rotational viscosity -4 eta_r V_i V_j F (I - ee) u_ij,
 *       u_ij = v_ij + 1/2 r_ij x (w_i + w_j); M5 + M6 reproduce the third and
 *       fifth terms of Eq. 2 for div v = 0.
 *   M7  local interaction F_sn = -C_l V_i V_j W u_ij between unlike species,
 *       with the reaction on the other species (Sec. 2.1).
 *   M8  spin torque tau_i = sum_j -1/2 r_ij x (f^rot_ij + f^sn_ij), so that
 *       orbital + spin angular momentum is conserved; I_i dw_i/dt = tau_i.
 *   M9  kick-drift-kick velocity Verlet; rigid rotating walls; periodic z.
 * Walls are viscous ("normal fluid") particles in every species test.
 *
 * Two optional steps of Algorithm 1 whose formulas the paper does not print,
 * in the reading stated in sph_oracle.h:
 *   pressure filter  Pf_i = sum_j V_j P_j W_ij / sum_j V_j W_ij over i itself
 *                    and its neighbours (outer walls excluded), applied right
 *                    after the equation of state;
 *   collision model  for a pair closer than col_dist whose distance shrinks
 *                    (r_ij . v_ij < 0), the impulse of a binary collision of
 *                    two spheres with restitution col_e along e = r_ij / r:
 *                    dv_i = -(1 + col_e) m_j / (m_i + m_j) (e . v_ij) e,
 *                    entered in the pair pass as the force m_i dv_i / dt.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>

static const double ORC_PI = 3.14159265358979323846;

static double alpha_D(const orc_params* p) {
  return 21.0 / (16.0 * ORC_PI * p->h * p->h * p->h);
}

double orc_W(const orc_params* p, double r) {
  double q = r / p->h;
  if (!(q < 2.0)) return 0.0;
  double t = 1.0 - 0.5 * q;
  double t2 = t * t;
  return alpha_D(p) * t2 * t2 * (2.0 * q + 1.0);
}

double orc_F(const orc_params* p, double r) {
  double q = r / p->h;
  if (!(q < 2.0)) return 0.0;
  double t = 1.0 - 0.5 * q;
  return 5.0 * alpha_D(p) * t * t * t / (p->h * p->h);
}

double orc_lattice_sum(const orc_params* p) {
  int m = (int)ceil(2.0 * p->h / p->dx) + 1;
  double s = 0.0;
  for (int a = -m; a <= m; ++a)
    for (int b = -m; b <= m; ++b)
      for (int c = -m; c <= m; ++c) {
        double r = p->dx * sqrt((double)(a * a + b * b + c * c));
        s += orc_W(p, r);
      }
  return s;
}

double orc_mass(const orc_params* p, int species) {
  double mn = p->rho0 / orc_lattice_sum(p);
  return species == 0 ? p->mass_ratio * mn : mn;
}

void orc_pair_delta(const orc_params* p, const double* ri, const double* rj, double d[3]) {
  d[0] = ri[0] - rj[0];
  d[1] = ri[1] - rj[1];
  d[2] = ri[2] - rj[2];
  if (p->periodic_z) {
    double half = 0.5 * p->Hz;
    if (d[2] > half) d[2] -= p->Hz;
    else if (d[2] < -half) d[2] += p->Hz;
  }
}

static double norm2(const double d[3]) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

static double cutoff2(const orc_params* p) { return (2.0 * p->h) * (2.0 * p->h); }

int64_t orc_neighbors(const orc_params* p, int64_t n, const double* pos,
                      int64_t* offsets, int64_t* nbr, int64_t cap) {
  double c2 = cutoff2(p);
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    offsets[i] = total;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      orc_pair_delta(p, pos + 3 * i, pos + 3 * j, d);
      if (norm2(d) < c2) {
        if (total < cap) nbr[total] = j;
        ++total;
      }
    }
  }
  offsets[n] = total;
  return total;
}

static double tait(const orc_params* p, double rho) {
  /* Eq. 4 */
  return p->p0 * pow(rho / p->rho0, p->alpha_P) - p->beta_P;
}

void orc_density(const orc_params* p, int64_t n, const double* pos,
                 const uint8_t* species, const int64_t* rows, int64_t nrows,
                 double* rho, double* P) {
  double c2 = cutoff2(p);
  double m_n = orc_mass(p, 1), m_s = orc_mass(p, 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nrows; ++k) {
    int64_t i = rows ? rows[k] : k;
    double r;
    if (species[i] == 3) {
      r = p->rho0;
    } else {
      r = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        double d[3];
        orc_pair_delta(p, pos + 3 * i, pos + 3 * j, d);
        double q2 = norm2(d);
        if (q2 < c2) r += (species[j] == 0 ? m_s : m_n) * orc_W(p, sqrt(q2));
      }
    }
    rho[i] = r;
    P[i] = tait(p, r);
  }
}

void orc_pressure_filter(const orc_params* p, int64_t n, const double* pos,
                         const uint8_t* species, const double* rho, const double* P,
                         const int64_t* rows, int64_t nrows, double* Pf) {
  double c2 = cutoff2(p);
  double m_n = orc_mass(p, 1), m_s = orc_mass(p, 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nrows; ++k) {
    int64_t i = rows ? rows[k] : k;
    if (species[i] == 3) {
      Pf[i] = P[i];
      continue;
    }
    double num = 0.0, den = 0.0;
    for (int64_t j = 0; j < n; ++j) { /* j = i gives the self term W(0) */
      if (species[j] == 3) continue;
      double d[3];
      orc_pair_delta(p, pos + 3 * i, pos + 3 * j, d);
      double q2 = norm2(d);
      if (!(q2 < c2)) continue;
      double Vj = (species[j] == 0 ? m_s : m_n) / rho[j];
      double w = Vj * orc_W(p, sqrt(q2));
      num += w * P[j];
      den += w;
    }
    Pf[i] = num / den;
  }
}

static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_forces_ex(const orc_params* p, int64_t n, const double* pos,
                   const double* vel, const double* spin, const uint8_t* species,
                   const double* rho, const double* P, const int64_t* rows,
                   int64_t nrows, double* acc, double* dspin, double* wall_T,
                   double* term_mag, double* scale) {
  double c2 = cutoff2(p);
  double m_n = orc_mass(p, 1), m_s = orc_mass(p, 0);
  double A = 10.0 * (p->eta_bar - 0.6 * p->eta_r); /* M5 */
  double col2 = p->col_dist * p->col_dist;          /* collision model */
  double B = 4.0 * p->eta_r;                       /* M6 */
  unsigned fl = p->flags;
  double mag[5] = {0, 0, 0, 0, 0};
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : mag[:5])
  for (int64_t k = 0; k < nrows; ++k) {
    int64_t i = rows ? rows[k] : k;
    double* ai = acc + 3 * i;
    double* bi = dspin + 3 * i;
    double* Ti = wall_T ? wall_T + 3 * i : NULL;
    ai[0] = ai[1] = ai[2] = 0.0;
    bi[0] = bi[1] = bi[2] = 0.0;
    if (Ti) Ti[0] = Ti[1] = Ti[2] = 0.0;
    if (scale) scale[2 * i] = scale[2 * i + 1] = 0.0;
    if (species[i] >= 2) continue; /* walls carry no dynamics */
    double mi = species[i] == 0 ? m_s : m_n;
    double Vi = mi / rho[i];
    double Pri = P[i] / (rho[i] * rho[i]);
    int inv_i = species[i] == 0;
    double fsum[6][3]; /* the five terms of M3-M7, then the collision force */
    memset(fsum, 0, sizeof fsum);
    double tau[3] = {0, 0, 0};
    double Tw[3] = {0, 0, 0};
    double fabs_sum = 0.0, tabs_sum = 0.0; /* sum_j |f_ij| and sum_j |tau_ij| */
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      orc_pair_delta(p, pos + 3 * i, pos + 3 * j, d);
      double r2 = norm2(d);
      if (!(r2 < c2) || !(r2 > 0.0)) continue;
      double r = sqrt(r2);
      double e[3] = {d[0] / r, d[1] / r, d[2] / r};
      double F = orc_F(p, r);
      double W = orc_W(p, r);
      double mj = species[j] == 0 ? m_s : m_n;
      double Vj = mj / rho[j];
      int inv_j = species[j] == 0;
      int chiX = inv_i != inv_j;
      int chiV = !inv_i && !inv_j;
      double f[6][3];
      memset(f, 0, sizeof f);
      /* M3 pressure */
      if (fl & ORC_TERM_P) {
        double s = mi * mj * (Pri + P[j] / (rho[j] * rho[j])) * F;
        f[0][0] = s * d[0];
        f[0][1] = s * d[1];
        f[0][2] = s * d[2];
      }
      /* M4 interfacial (temperature-gradient) force */
      if ((fl & ORC_TERM_T) && chiX) {
        double s = p->C_T * Vi * Vj * F;
        f[1][0] = s * d[0];
        f[1][1] = s * d[1];
        f[1][2] = (fl & ORC_HPROJ) ? 0.0 : s * d[2];
      }
      double vij[3] = {vel[3 * i] - vel[3 * j], vel[3 * i + 1] - vel[3 * j + 1],
                       vel[3 * i + 2] - vel[3 * j + 2]};
      double ws[3] = {spin[3 * i] + spin[3 * j], spin[3 * i + 1] + spin[3 * j + 1],
                      spin[3 * i + 2] + spin[3 * j + 2]};
      double dxw[3];
      cross(d, ws, dxw);
      double u[3] = {vij[0] + 0.5 * dxw[0], vij[1] + 0.5 * dxw[1], vij[2] + 0.5 * dxw[2]};
      /* M5 central shear viscosity */
      if ((fl & ORC_TERM_SH) && chiV) {
        double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
        double s = -A * Vi * Vj * F * ev;
        f[2][0] = s * e[0];
        f[2][1] = s * e[1];
        f[2][2] = s * e[2];
      }
      /* M6 transverse rotational viscosity with spin */
      if ((fl & ORC_TERM_ROT) && chiV) {
        double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        double s = -B * Vi * Vj * F;
        f[3][0] = s * (u[0] - eu * e[0]);
        f[3][1] = s * (u[1] - eu * e[1]);
        f[3][2] = s * (u[2] - eu * e[2]);
      }
      /* M7 local interaction */
      if ((fl & ORC_TERM_SN) && chiX) {
        const double* w = (fl & ORC_SN_LITERAL) ? vij : u;
        double s = -p->C_l * Vi * Vj * W;
        f[4][0] = s * w[0];
        f[4][1] = s * w[1];
        f[4][2] = s * w[2];
      }
      /* collision model: approaching pair closer than col_dist */
      if ((fl & ORC_COLLISION) && r2 < col2) {
        double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
        if (ev < 0.0) {
          double s = -(1.0 + p->col_e) * (mi * mj / (mi + mj)) * ev / p->dt;
          f[5][0] = s * e[0];
          f[5][1] = s * e[1];
          f[5][2] = s * e[2];
        }
      }
      /* M8 spin torque */
      double fs[3] = {f[3][0], f[3][1], f[3][2]};
      if (!(fl & ORC_SN_LITERAL)) {
        fs[0] += f[4][0];
        fs[1] += f[4][1];
        fs[2] += f[4][2];
      }
      double t[3];
      cross(d, fs, t);
      t[0] *= -0.5;
      t[1] *= -0.5;
      t[2] *= -0.5;
      for (int a = 0; a < 3; ++a) tau[a] += t[a];
      for (int q = 0; q < 6; ++q)
        for (int a = 0; a < 3; ++a) fsum[q][a] += f[q][a];
      if (scale) {
        double fp[3];
        for (int a = 0; a < 3; ++a)
          fp[a] = f[0][a] + f[1][a] + f[2][a] + f[3][a] + f[4][a] + f[5][a];
        fabs_sum += sqrt(norm2(fp));
        tabs_sum += sqrt(norm2(t));
      }
      if (species[j] >= 2) {
        double ft[3] = {f[0][0] + f[1][0] + f[2][0] + f[3][0] + f[4][0] + f[5][0],
                        f[0][1] + f[1][1] + f[2][1] + f[3][1] + f[4][1] + f[5][1],
                        f[0][2] + f[1][2] + f[2][2] + f[3][2] + f[4][2] + f[5][2]};
        double o[3];
        cross(pos + 3 * i, ft, o);
        for (int a = 0; a < 3; ++a) Tw[a] += o[a] + t[a];
      }
    }
    double Ii = p->inertia_coef * mi * p->dx * p->dx;
    for (int a = 0; a < 3; ++a) {
      double ft = fsum[0][a] + fsum[1][a] + fsum[2][a] + fsum[3][a] + fsum[4][a] + fsum[5][a];
      ai[a] = ft / mi;
      bi[a] = tau[a] / Ii;
      if (Ti) Ti[a] = Tw[a];
    }
    if (scale) {
      scale[2 * i] = fabs_sum / mi;
      scale[2 * i + 1] = tabs_sum / Ii;
    }
    for (int q = 0; q < 5; ++q)
      mag[q] += sqrt(fsum[q][0] * fsum[q][0] + fsum[q][1] * fsum[q][1] +
                     fsum[q][2] * fsum[q][2]);
  }
  if (term_mag)
    for (int q = 0; q < 5; ++q) term_mag[q] += mag[q];
}

void orc_forces(const orc_params* p, int64_t n, const double* pos,
                const double* vel, const double* spin, const uint8_t* species,
                const double* rho, const double* P, const int64_t* rows,
                int64_t nrows, double* acc, double* dspin, double* wall_T,
                double* term_mag) {
  orc_forces_ex(p, n, pos, vel, spin, species, rho, P, rows, nrows, acc, dspin, wall_T,
                term_mag, NULL);
}

void orc_place_walls(const orc_params* p, int64_t n, const uint8_t* species,
                     const double* wall_ref, double theta, double* pos,
                     double* vel, double* spin) {
  double c = cos(theta), s = sin(theta);
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] < 2) continue;
    double x0 = wall_ref[3 * i], y0 = wall_ref[3 * i + 1];
    double x = c * x0 - s * y0;
    double y = s * x0 + c * y0;
    pos[3 * i] = x;
    pos[3 * i + 1] = y;
    pos[3 * i + 2] = wall_ref[3 * i + 2];
    vel[3 * i] = -p->Omega * y;
    vel[3 * i + 1] = p->Omega * x;
    vel[3 * i + 2] = 0.0;
    spin[3 * i] = 0.0;
    spin[3 * i + 1] = 0.0;
    spin[3 * i + 2] = p->Omega;
  }
}

static void sum_wall_torque(int64_t n, const uint8_t* species, const double* wT, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] >= 2) continue;
    out[0] += wT[3 * i];
    out[1] += wT[3 * i + 1];
    out[2] += wT[3 * i + 2];
  }
}

#include <stdlib.h>

static void evaluate(const orc_params* p, int64_t n, const double* pos,
                     const double* vel, const double* spin, const uint8_t* species,
                     double* rho, double* P, double* acc, double* dspin,
                     double* T_wall_sum) {
  orc_density(p, n, pos, species, NULL, n, rho, P);
  if (p->flags & ORC_PFILTER) {
    double* Pf = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_pressure_filter(p, n, pos, species, rho, P, NULL, n, Pf);
    memcpy(P, Pf, sizeof(double) * (size_t)n);
    free(Pf);
  }
  double* wT = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  orc_forces(p, n, pos, vel, spin, species, rho, P, NULL, n, acc, dspin, wT, NULL);
  sum_wall_torque(n, species, wT, T_wall_sum);
  free(wT);
}

void orc_init(const orc_params* p, int64_t n, double* pos, double* vel,
              double* spin, const uint8_t* species, const double* wall_ref,
              double theta, double* rho, double* P, double* acc, double* dspin,
              double* T_wall_sum) {
  orc_place_walls(p, n, species, wall_ref, theta, pos, vel, spin);
  evaluate(p, n, pos, vel, spin, species, rho, P, acc, dspin, T_wall_sum);
}

void orc_step(const orc_params* p, int64_t n, double* pos, double* vel,
              double* spin, const uint8_t* species, const double* wall_ref,
              double* theta, double* rho, double* P, double* acc, double* dspin,
              double* T_wall_sum, double* J_wall) {
  double hdt = 0.5 * p->dt;
  /* kick (half step) and drift, fluid only */
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] >= 2) continue;
    for (int a = 0; a < 3; ++a) {
      vel[3 * i + a] += hdt * acc[3 * i + a];
      spin[3 * i + a] += hdt * dspin[3 * i + a];
      pos[3 * i + a] += p->dt * vel[3 * i + a];
    }
    if (p->periodic_z) {
      if (pos[3 * i + 2] >= p->Hz) pos[3 * i + 2] -= p->Hz;
      else if (pos[3 * i + 2] < 0.0) pos[3 * i + 2] += p->Hz;
    }
  }
  /* rigid vessel: advance the wall phase in FP64 and place the walls */
  *theta += p->Omega * p->dt;
  orc_place_walls(p, n, species, wall_ref, *theta, pos, vel, spin);
  /* density, pressure, forces at the new positions with half-step v, w */
  double T_old[3] = {T_wall_sum[0], T_wall_sum[1], T_wall_sum[2]};
  evaluate(p, n, pos, vel, spin, species, rho, P, acc, dspin, T_wall_sum);
  /* second half kick */
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] >= 2) continue;
    for (int a = 0; a < 3; ++a) {
      vel[3 * i + a] += hdt * acc[3 * i + a];
      spin[3 * i + a] += hdt * dspin[3 * i + a];
    }
  }
  for (int a = 0; a < 3; ++a) J_wall[a] += hdt * (T_old[a] + T_wall_sum[a]);
}

static double internal_energy(const orc_params* p, double rho) {
  /* e(rho) = int_{rho0}^{rho} P(s)/s^2 ds for the Tait law of Eq. 4 */
  double a = p->alpha_P;
  return p->p0 / ((a - 1.0) * p->rho0) * (pow(rho / p->rho0, a - 1.0) - 1.0) +
         p->beta_P * (1.0 / rho - 1.0 / p->rho0);
}

void orc_diagnostics(const orc_params* p, int64_t n, const double* pos,
                     const double* vel, const double* spin,
                     const uint8_t* species, const double* rho,
                     const double* T_wall_sum, const double* J_wall,
                     orc_diag* out) {
  memset(out, 0, sizeof *out);
  out->rho_min = INFINITY;
  out->rho_max = -INFINITY;
  double c2 = cutoff2(p);
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] >= 2) continue;
    double m = orc_mass(p, species[i]);
    double I = p->inertia_coef * m * p->dx * p->dx;
    const double* r = pos + 3 * i;
    const double* v = vel + 3 * i;
    const double* w = spin + 3 * i;
    out->mass += m;
    if (species[i] == 0) out->mass_s += m;
    else out->mass_n += m;
    double L[3];
    cross(r, v, L);
    for (int a = 0; a < 3; ++a) {
      out->mom[a] += m * v[a];
      out->L_orb[a] += m * L[a];
      out->L_spin[a] += I * w[a];
    }
    double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    out->E_kin += 0.5 * m * v2;
    out->E_rot += 0.5 * I * ((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2]);
    out->E_int += m * internal_energy(p, rho[i]);
    if (rho[i] < out->rho_min) out->rho_min = rho[i];
    if (rho[i] > out->rho_max) out->rho_max = rho[i];
    if (sqrt(v2) > out->v_max) out->v_max = sqrt(v2);
  }
  int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] >= 2) continue; /* pairs of the fluid rows (force pass) */
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      orc_pair_delta(p, pos + 3 * i, pos + 3 * j, d);
      if (norm2(d) < c2) ++pairs;
    }
  }
  out->n_pairs = pairs;
  for (int a = 0; a < 3; ++a) {
    out->T_wall[a] = T_wall_sum ? T_wall_sum[a] : 0.0;
    out->J_wall[a] = J_wall ? J_wall[a] : 0.0;
  }
}
