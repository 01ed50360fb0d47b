/*
 * CPU FP64 oracle of the two-fluid spin-SPH time step (test infrastructure).
 *
 * This is the slow, obviously-correct reference that the CUDA library is
 * checked against.  It is used only by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; the product path never calls it.  It
 * shares no code, header or constant with the CUDA library.
 *
 * Every pair loop is a plain O(N^2) double loop over j = 0..n-1 in ascending
 * order; there is no cell list, no blocking and no reordering.
 *
 * Species codes: 0 inviscid, 1 viscous, 2 inner wall, 3 outer wall.
 * Arrays of vectors are xyz-interleaved (3n doubles).
 *
 * Parity status: every function below is pinned by tests/test_oracle_pins.py
 * (kernel normalisation by quadrature, lattice rest density, also with
 * unequal species masses, momentum and angular-momentum conservation
 * (also at a lattice spacing other than 1, which fixes the dx^2 of the spin
 * inertia in both the torque update and the diagnostics),
 * rigid-rotation zero viscous force, also next to the rotating walls,
 * continuum limit of the viscous/spin terms, energy conservation, the
 * diagnostics' energies against the momenta of uniform states, brute-force
 * neighbour sets against a k-d tree, time reversibility of the integrator).  The
 * interfacial force is pinned in sign, projection, reaction and scale: on a
 * lattice split by a species interface its summed force per unit area is
 * the closed form of the kernel's second moment, -C_T/2 in the continuum.
 * The values of C_T and C_l themselves are free parameters (the paper
 * prints the continuum form of the two forces only); the local-interaction
 * magnitude is pinned in sign, direction and reaction only.
 *
 * The pressure filter and the collision model are named in Algorithm 1 but
 * their formulas are not printed; they follow a reading (a zeroth-order
 * kernel average of P; a binary inelastic collision along the line of
 * centres of approaching pairs closer than col_dist, with restitution col_e,
 * applied as the acceleration that gives that velocity change over one
 * step).  The reading is pinned by closed forms and invariants (constant and
 * linear fields, the spike response on the lattice, the two-body collision
 * law, momentum and angular-momentum conservation); whether it is the
 * paper's own form cannot be checked.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_TERM_P = 1u,       /* Tait pressure gradient                      */
  ORC_TERM_T = 2u,       /* interfacial (temperature-gradient) force     */
  ORC_TERM_SH = 4u,      /* central shear viscosity                      */
  ORC_TERM_ROT = 8u,     /* transverse rotational viscosity with spin    */
  ORC_TERM_SN = 16u,     /* local interaction force F_sn                 */
  ORC_HPROJ = 32u,       /* interfacial force acts horizontally only     */
  ORC_SN_LITERAL = 64u,  /* F_sn on plain v_ij (no spin coupling/torque) */
  ORC_PFILTER = 128u,    /* pressure filter after the equation of state  */
  ORC_COLLISION = 256u,  /* collision model in the pair pass             */
  ORC_TERMS_ALL = 31u
};

typedef struct {
  double dx, h, rho0;
  double alpha_P, p0, beta_P;      /* Eq. 4: P = p0 (rho/rho0)^alpha_P - beta_P */
  double eta_bar, eta_r, xi_bar;   /* shear, rotational, bulk viscosity (Eq. 2) */
  double C_l;                      /* local interaction coefficient            */
  double C_T;                      /* signed interfacial coefficient           */
  double C_omega;                  /* recorded, not applied                    */
  double mass_ratio;               /* m_s / m_n                                */
  double inertia_coef;             /* I_i = inertia_coef m_i dx^2              */
  double Omega, dt;
  double col_dist;                 /* collision model: pair distance below     */
  double col_e;                    /*   which approaching pairs collide, and   */
                                   /*   the restitution coefficient            */
  double Hz;                       /* z period                                 */
  int periodic_z;
  unsigned flags;
} orc_params;

typedef struct {
  double mass, mass_s, mass_n;
  double mom[3];
  double L_orb[3], L_spin[3];
  double E_kin, E_rot, E_int;
  double T_wall[3];                /* torque of the walls on the fluid now     */
  double J_wall[3];                /* time integral of T_wall                  */
  double rho_min, rho_max, v_max;
  int64_t n_pairs;                 /* ordered pairs (i fluid, j != i, r < 2h)  */
} orc_diag;

/* Wendland C2 kernel W(r) and F(r) = -(1/r) dW/dr, support 2h. */
double orc_W(const orc_params* p, double r);
double orc_F(const orc_params* p, double r);
/* Sum of W(|n| dx) over the integer lattice n in Z^3. */
double orc_lattice_sum(const orc_params* p);
/* Particle mass m_n = rho0 / lattice_sum; m_s = mass_ratio m_n; walls m_n. */
double orc_mass(const orc_params* p, int species);

/* Pair vector r_i - r_j with the minimum image in z when periodic. */
void orc_pair_delta(const orc_params* p, const double* ri, const double* rj, double d[3]);

/* Brute-force neighbour lists: j != i with r^2 < (2h)^2.  offsets has n+1
 * entries; nbr receives at most cap indices; returns the total count. */
int64_t orc_neighbors(const orc_params* p, int64_t n, const double* pos,
                      int64_t* offsets, int64_t* nbr, int64_t cap);

/* Density (summation, self included) and Tait pressure for the listed rows. */
void orc_density(const orc_params* p, int64_t n, const double* pos,
                 const uint8_t* species, const int64_t* rows, int64_t nrows,
                 double* rho, double* P);

/* Pressure filter (Algorithm 1, after the equation of state) for the listed
 * rows: the kernel-weighted volume average of the pressure,
 *   Pf_i = sum_j V_j P_j W_ij / sum_j V_j W_ij,  V_j = m_j / rho_j,
 * over j = i and the neighbours r < 2h of i, outer-wall particles excluded
 * (their pressure is not computed); outer-wall rows keep their P.  rho and P
 * are read for every particle. */
void orc_pressure_filter(const orc_params* p, int64_t n, const double* pos,
                         const uint8_t* species, const double* rho, const double* P,
                         const int64_t* rows, int64_t nrows, double* Pf);

/* Pair forces for the listed rows: acc = f/m, dspin = tau/I; wall_T receives
 * the torque (orbital about the z axis + spin) exerted by wall neighbours.
 * term_mag (optional, 5 doubles) accumulates sum_i |f_i^term| per term
 * (the collision force, when on, is not one of the five). */
void orc_forces(const orc_params* p, int64_t n, const double* pos,
                const double* vel, const double* spin, const uint8_t* species,
                const double* rho, const double* P, const int64_t* rows,
                int64_t nrows, double* acc, double* dspin, double* wall_T,
                double* term_mag);

/* orc_forces, and (scale, optional, 2 doubles per particle) for each listed
 * fluid row the scale of its absolute pair sums: sum_j |f_ij| / m_i and
 * sum_j |tau_ij| / I_i, with f_ij the whole pair force and tau_ij the pair's
 * spin torque (0 for wall rows).  A summation in another order can change
 * acc_i and dspin_i only by rounding relative to these sums. */
void orc_forces_ex(const orc_params* p, int64_t n, const double* pos,
                   const double* vel, const double* spin, const uint8_t* species,
                   const double* rho, const double* P, const int64_t* rows,
                   int64_t nrows, double* acc, double* dspin, double* wall_T,
                   double* term_mag, double* scale);

/* Place the rigid walls at phase theta from their reference positions. */
void orc_place_walls(const orc_params* p, int64_t n, const uint8_t* species,
                     const double* wall_ref, double theta, double* pos,
                     double* vel, double* spin);

/* Initial evaluation: walls at theta, density (+ the pressure filter when
 * on), forces (a_0, alpha_0). */
void orc_init(const orc_params* p, int64_t n, double* pos, double* vel,
              double* spin, const uint8_t* species, const double* wall_ref,
              double theta, double* rho, double* P, double* acc, double* dspin,
              double* T_wall_sum);

/* One kick-drift-kick velocity Verlet step (Algorithm 1 inner body). */
void orc_step(const orc_params* p, int64_t n, double* pos, double* vel,
              double* spin, const uint8_t* species, const double* wall_ref,
              double* theta, double* rho, double* P, double* acc, double* dspin,
              double* T_wall_sum, double* J_wall);

/* FP64 conservation diagnostics over the fluid particles. */
void orc_diagnostics(const orc_params* p, int64_t n, const double* pos,
                     const double* vel, const double* spin,
                     const uint8_t* species, const double* rho,
                     const double* T_wall_sum, const double* J_wall,
                     orc_diag* out);

#ifdef __cplusplus
}
#endif
#endif
