// Internal declarations shared by the translation units of libsps.
// Data layout in HBM (per context):
//   geometry   pos (N x 3), rad (N) FP64; nodes X, normals Nrm as 3 planes of
//              NP = N*P, weights W (NP); FP32 copies for the mixed far field.
//   near lists CSR by target sphere (near_ptr N+1, near_idx sorted ascending).
//   surface fields 3 planes of NP (FP64).
//   VSH        coef: N x NR rows, NR = 6*NC real numbers per sphere
//              (type V/W/X, n, m >= 0, re/im), the multipliers of eq. rhoshexp.
//   near field per source sphere, E = (L+1)(L+2)/2 entries (n', m' >= 0,
//              n' <= L = p+2, m'-major) x F fields, complex.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/sps.h"

#define SPS_PI 3.14159265358979323846

namespace sps {

constexpr int kFieldsK = 25;   // fields summed per target for the traction
constexpr int kFieldsS = 10;   // fields summed per target for the velocity
constexpr int kMaxP = 16;
// near entries closer than this many source radii from the source centre are
// evaluated in FP64 in the mixed path (the VSH terms decay slowly there)
#ifndef SPS_CLOSE_RADIUS
#define SPS_CLOSE_RADIUS 1.5
#endif
constexpr double kCloseRadius = SPS_CLOSE_RADIUS;

struct Tables {
  int p = 0, P = 0, NC = 0, NR = 0, L = 0, E = 0;
  std::vector<double> t, wgl;             // Gauss-Legendre nodes / weights
  std::vector<double> unit_nrm;           // 3 planes of P
  std::vector<double> unit_w;             // P
  std::vector<double> anal;               // NR x 3P, row-major
  std::vector<double> synth;              // 3P x NR, row-major
  std::vector<double> multS, multK;       // NR (per row: self multipliers)
  std::vector<double> kappa;              // NC: phi_nm = kappa * H_n^m
  std::vector<double> potfac;             // (p+1) x 6: near-field potential factors per degree
};
void build_tables(int p, Tables& T);

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace sps

// Planar walls (Sec. 3.3.3 particle-boundary constraints): plane n.x = d with
// a unit normal n pointing into the fluid, row (n_x, n_y, n_z, d)
constexpr int kMaxWalls = 8;
struct SpsWalls {
  int n = 0;
  double w[kMaxWalls][4] = {};
};

struct sps_ctx {
  sps_params prm;
  SpsWalls walls;
  // phase timers
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_rec;
  size_t ev_used = 0;
  cudaStream_t stream = nullptr;
  sps::Tables T;
  std::string err;
  long long launches = 0;

  // unit tables on device
  double *d_unit_nrm = nullptr, *d_unit_w = nullptr;
  double *d_anal = nullptr;     // NR x 3P row-major analysis
  double *d_synthS = nullptr;   // 3P x NR row-major synthesis * multS
  double *d_synthK = nullptr;   // 3P x NR row-major synthesis * multK
  double *d_kappa = nullptr, *d_potfac = nullptr;
  // near-field coefficient map as sparse matrices (per field set K / S):
  // fcoef_s = FM coef_s  (rows 2*E*F, cols NR) and its transpose
  struct Sparse {
    int rows = 0, cols = 0, nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double* v = nullptr;
  } fmK, fmS, fmKt, fmSt;
  // transposed self matrices for the adjoint
  double *d_analT = nullptr;    // 3P x NR row-major (analysis transposed)
  double *d_synthST = nullptr;  // NR x 3P (synthesis * multS, transposed)
  double *d_synthKT = nullptr;  // NR x 3P
  double *d_coefbar = nullptr;  // N x NR adjoint of the VSH coefficients
  double *d_ebar = nullptr;     // N x E x kFieldsK x 2 adjoint of the field coefficients
  double *d_sigtot = nullptr, *d_ubar = nullptr, *d_sbar = nullptr, *d_lam = nullptr, *d_rbar = nullptr;
  bool adjoint_mode = false;    // GMRES applies A^T instead of A
  long long layer_applies = 0;  // layer-operator applications since creation
  long long stats_layer0 = 0;   // ... at the start of the current API call
  float *d_anal32 = nullptr, *d_synthS32 = nullptr, *d_synthK32 = nullptr;
  // tensor-core transforms (mixed path): matrices split into three BF16 terms
  // in the layout of k_sht_tc; analysis, synthesis x multS, synthesis x multK
  struct TcMat {
    uint16_t* d = nullptr;
    int R = 0, C = 0, Kpad = 0;
  } tcA, tcS, tcK;
  int* d_tcflag = nullptr;       // set by a tensor-core transform that timed out
  uint16_t* d_tcsplit = nullptr; // the transform input split into BF16 terms, chunk layout
  size_t cap_tcsplit = 0;

  // geometry
  int N = 0, NP = 0, capN = 0;
  double *d_pos = nullptr, *d_rad = nullptr;
  double *d_X = nullptr, *d_Nrm = nullptr, *d_W = nullptr;
  float *d_rel32 = nullptr, *d_N32 = nullptr, *d_W32 = nullptr;  // node - own centre, normal, w
  float *d_chi = nullptr, *d_clo = nullptr;                       // centres as hi + lo (N x 3)
  int *d_near_ptr = nullptr, *d_near_idx = nullptr;
  int n_near = 0, cap_near = 0;
  // source-major near field (mixed path): reverse index and per-pair centre
  // offsets (see k_near_rev), per-(pair, node) results (3 planes of n_near P)
  int *d_near_rev = nullptr;
  float *d_near_geo = nullptr;
  double *d_near_buf = nullptr;
  size_t cap_near_rev = 0, cap_near_geo = 0, cap_near_buf = 0;
  // close near entries (mixed path FP64 list): nodes, CSR into source spheres
  int n_close = 0, n_close_src = 0;
  int *d_close_node = nullptr, *d_close_ptr = nullptr, *d_close_src = nullptr;
  size_t cap_close_node = 0, cap_close_ptr = 0, cap_close_src = 0;
  bool have_geom = false;

  // operator scratch
  double *d_coef = nullptr;      // N x NR
  double *d_fcoef = nullptr;     // N x E x kFieldsK x 2
  float *d_fcoef32 = nullptr;    // the same rounded to FP32 (mixed near field)
  float2 *d_fcoefdw = nullptr;   // the same as FP32 hi + lo pairs (close entries)
  double *d_mom = nullptr;       // N x 6 (per-sphere moments)
  double *d_tmp3 = nullptr;      // 3NP scratch
  float *d_sig32 = nullptr;      // 3NP FP32 w*sigma for the mixed far field
  double *d_part = nullptr;      // far-field partial sums (splits x 3NP)
  size_t cap_part = 0;
  float4 *d_dwsrc = nullptr;     // double-float far field: 3 x NP staged source values
  size_t cap_dwsrc = 0;
  // grid orientation (Sec. 5.4): rotation Q_i per sphere (N x 9, row-major),
  // in force while rot_n equals the number of spheres; densities rotated
  // into the sphere frames for the VSH transforms
  double *d_rot = nullptr;
  size_t cap_rot = 0;
  int rot_n = 0;
  double *d_sigloc = nullptr;    // 3NP: a density in the sphere frames
  size_t cap_sigloc = 0;

  // GMRES
  int gm_cap_n = 0, gm_cap_k = 0;
  double *d_Q = nullptr;         // (k+1) x n Krylov basis
  double *d_w = nullptr, *d_h = nullptr, *d_red = nullptr;
  double *h_pinned = nullptr;    // pinned host scratch for scalars
  double *d_sc = nullptr;        // fixed scratch of sps_dot (partials + results), from sps_create
  double *d_rho = nullptr, *d_zeta = nullptr, *d_b = nullptr, *d_u = nullptr;
  double *d_zeta_nc = nullptr;   // density of the last U_nc solve (warm start)
  long long zeta_nc_n = 0;       // node count it belongs to (0: none)
  long long zeta_n = 0;          // node count of the last sps_mobility_apply density in d_zeta
  double *d_r = nullptr, *d_dz = nullptr;
  // solve history of one collision step (initial guesses): orthonormal
  // right-hand sides and matching solution combinations
  double *d_Pb = nullptr, *d_Px = nullptr;
  long long proj_n = 0;
  int proj_m = 0, proj_old = 0;   // columns in use, oldest column once full
  bool proj_on = false;
  // the previous collision step's contact pairs and gamma (initial guess of
  // Algorithm 1 with bb_warm)
  int *d_prev_ij = nullptr;
  double *d_prev_gam = nullptr;
  size_t cap_prev_ij = 0, cap_prev_gam = 0;
  int prev_nc = 0, prev_N = 0;
  double prev_alpha = 0.0;       // bb_warm = 2: the previous step's last BB step length (0: none)
  double bb_alpha_last = 0.0;    // the step length Algorithm 1 used last

  // contacts
  int n_c = 0, cap_c = 0, c_N = 0;   // contacts, capacity, spheres they refer to
  int n_pair = 0;                // sphere-pair contacts (the first n_pair); the rest are wall contacts
  int prev_npair = 0;            // the same count of the previous step's list (bb_warm)
  int *d_wcount = nullptr;       // N+1: wall contacts per sphere, then their offsets
  int *d_wptr = nullptr;
  size_t cap_wcount = 0, cap_wptr = 0;
  int *d_inc_fill = nullptr;     // N+1 fill counters of the incidence transpose
  int *d_cl_fill = nullptr;      // cells + 1 fill counters of the cell counting sort
  int *d_scan_tot = nullptr;     // block totals of sps_exclusive_scan
  size_t cap_inc_fill = 0, cap_cl_fill = 0, cap_scan_tot = 0;
  int *d_cij = nullptr;          // n_c x 2
  double *d_cphi = nullptr, *d_cn = nullptr;
  int *d_ccount = nullptr, *d_cptr = nullptr;  // N+1
  int *d_inc_ptr = nullptr, *d_inc = nullptr;  // incidence CSR by sphere (2 n_c)
  void *d_cub = nullptr; size_t cub_bytes = 0;
  int *d_keys = nullptr, *d_vals = nullptr, *d_keys2 = nullptr, *d_vals2 = nullptr;
  int *d_ccount2 = nullptr, *d_inc_cnt = nullptr;  // N+1: contacts as second sphere, incidences
  size_t cap_cnt = 0;
  // cell list of the contact search: keys / sphere ids (and sorted copies),
  // per-cell [first, end) into the sorted order, sorted FP32 / FP64 copies of
  // (x, y, z, a); bounds partials
  int *d_cl_key = nullptr, *d_cl_id = nullptr, *d_cl_key2 = nullptr, *d_cl_id2 = nullptr;
  int *d_cl_range = nullptr;
  float4 *d_cl_f = nullptr;
  double4_32a *d_cl_d = nullptr;
  double *d_cl_part = nullptr;
  size_t cap_cl = 0, cap_cl_cells = 0;
  int *d_flag = nullptr;         // one int (input checks, counts)

  // BBPGD vectors (n_c each)
  double *d_gam = nullptr, *d_g = nullptr, *d_gam_new = nullptr, *d_g_new = nullptr;
  double *d_q = nullptr, *d_Mg = nullptr;
  double *d_FT = nullptr, *d_Unc = nullptr, *d_Uc = nullptr;
  int cap_bb = 0;
  double *d_bbpart = nullptr;    // BBPGD statistic partials (5 x blocks)
  double *d_apgd = nullptr;      // APGD: y, M y, scratch (n_c each) and reduction partials
  size_t cap_apgd = 0;
  double *d_gam_best = nullptr, *d_aux_best = nullptr;  // smallest-residual BBPGD iterate
  size_t cap_gam_best = 0, cap_aux_best = 0;
  // identity mobility: contact forces (N x 3), FT / U_nc / U_c (N x 6)
  double *d_F3 = nullptr, *d_iFT = nullptr;
  double *d_adj6a = nullptr, *d_adj6b = nullptr, *d_adjc = nullptr;  // collision adjoint scratch
  size_t cap_adj6 = 0, cap_adjc = 0;
  int *d_order = nullptr;        // spheres by block-local incident-contact count
  size_t cap_order = 0;
  bool order_valid = false;
  size_t cap_ident = 0;
};

// far field of an FP64-class application (fp32 = false) in double-float
// arithmetic: the SPS_FP64_DW path, or the mixed path's refinement with ir_dw
inline bool sps_far_dw(const sps_ctx* c) {
  return c->prm.precision == SPS_FP64_DW || (c->prm.precision == SPS_MIXED && c->prm.ir_dw);
}

// the per-sphere grid rotations in force for the current geometry, or null
inline const double* sps_rot(const sps_ctx* c) {
  return (c->rot_n > 0 && c->rot_n == c->N && c->have_geom) ? c->d_rot : nullptr;
}

// v <- Q^T v and v <- Q v for a row-major 3 x 3 rotation Q (an identity Q
// returns v unchanged to the bit: its zero products vanish exactly)
template <typename T, typename M>
__device__ __forceinline__ void sps_rot_t(const M* Q, T& x, T& y, T& z) {
  const T a = (T)Q[0] * x + (T)Q[3] * y + (T)Q[6] * z;
  const T b = (T)Q[1] * x + (T)Q[4] * y + (T)Q[7] * z;
  const T c = (T)Q[2] * x + (T)Q[5] * y + (T)Q[8] * z;
  x = a;
  y = b;
  z = c;
}
template <typename T, typename M>
__device__ __forceinline__ void sps_rot_n(const M* Q, T& x, T& y, T& z) {
  const T a = (T)Q[0] * x + (T)Q[1] * y + (T)Q[2] * z;
  const T b = (T)Q[3] * x + (T)Q[4] * y + (T)Q[5] * z;
  const T c = (T)Q[6] * x + (T)Q[7] * y + (T)Q[8] * z;
  x = a;
  y = b;
  z = c;
}

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
int sps_fail(sps_ctx* ctx, int code, const std::string& msg);
#define SPS_CUDA(ctx, call)                                                   \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return sps_fail(ctx, SPS_ERR_CUDA,                                      \
                      std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)
#define SPS_LAUNCHED(ctx)                                                     \
  do {                                                                        \
    (ctx)->launches++;                                                        \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess)                                                    \
      return sps_fail(ctx, SPS_ERR_CUDA,                                      \
                      std::string("launch: ") + cudaGetErrorString(e_));      \
  } while (0)
#define SPS_TRY(x)            \
  do {                        \
    int rc_ = (x);            \
    if (rc_ != SPS_OK) return rc_; \
  } while (0)

template <class T>
int sps_grow(sps_ctx* ctx, T** p, size_t& cap_elems, size_t need_elems) {
  if (need_elems <= cap_elems && *p) return SPS_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  size_t n = need_elems ? need_elems : 1;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    cap_elems = 0;
    return sps_fail(ctx, SPS_ERR_OOM, "cudaMalloc failed");
  }
  cap_elems = n;
  return SPS_OK;
}

// squared distance of a target (gx, gy, gz) from the centre of sphere j in
// units of a_j (ia = 1/a_j), evaluated identically wherever near entries are
// split into FP32 and FP64 ones
__device__ __forceinline__ double sps_close_r2(const double* pos, double ia, double gx, double gy,
                                               double gz, int j) {
  const double x = (gx - pos[3 * j]) * ia, y = (gy - pos[3 * j + 1]) * ia, z = (gz - pos[3 * j + 2]) * ia;
  return x * x + y * y + z * z;
}

// Contact test of Sec. 3.2 on loaded values: Phi = (d - R_i) - R_j <= delta_l
// with R = a_c_scale * a, delta_l = delta + drel (a_i + a_j) (drel = 0.3 is the
// paper's 30% of the sum of the radii) and every operation rounded
// separately, so that the all-pairs and the cell-list searches produce the
// same list to the bit.
struct SpsContactGeom {
  double phi, nx, ny, nz;
};

// Wall contact test on loaded values: Phi = (n . c - d) - a acs with
// n . c = (n_x x + n_y y) + n_z z, threshold delta + drel a, every operation
// rounded separately (the same list to the bit wherever it is evaluated)
__device__ __forceinline__ bool sps_wall_test(const double* wl, double x, double y, double z, double a,
                                              double acs, double delta, double drel, double* phi) {
  const double h = __dadd_rn(__dadd_rn(__dmul_rn(wl[0], x), __dmul_rn(wl[1], y)), __dmul_rn(wl[2], z));
  const double ph = __dsub_rn(__dsub_rn(h, wl[3]), __dmul_rn(a, acs));
  *phi = ph;
  return ph <= __dadd_rn(delta, __dmul_rn(drel, a));
}
__device__ __forceinline__ bool sps_contact_test(double xi, double yi, double zi, double ai, double xj,
                                                 double yj, double zj, double aj, double acs,
                                                 double delta, double drel, SpsContactGeom* g) {
  const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double d = __dsqrt_rn(d2);
  const double Ri = __dmul_rn(ai, acs), Rj = __dmul_rn(aj, acs);
  const double phi = __dsub_rn(__dsub_rn(d, Ri), Rj);
  const double dl = __dadd_rn(delta, __dmul_rn(drel, __dadd_rn(ai, aj)));
  if (!(phi <= dl)) return false;
  if (g) {
    g->phi = phi;
    g->nx = __ddiv_rn(dx, d);
    g->ny = __ddiv_rn(dy, d);
    g->nz = __ddiv_rn(dz, d);
  }
  return true;
}

// RAII phase timer: records an event pair around the enclosed launches
struct SpsPhase {
  sps_ctx* c;
  int ph;
  cudaEvent_t b = nullptr, e = nullptr;
  SpsPhase(sps_ctx* ctx, int phase);
  ~SpsPhase();
};

// ---------------------------------------------------------------------------
// launchers (each returns an sps_status)
// ---------------------------------------------------------------------------
// geometry / contacts (sps_geometry.cu)
int sps_launch_grid(sps_ctx* ctx);
// out = Q_i^T in (transpose) or Q_i in per node, 3 planes of NP (may alias)
int sps_launch_rotate(sps_ctx* ctx, const double* in, double* out, bool transpose);
int sps_launch_near_lists(sps_ctx* ctx);
int sps_launch_close_lists(sps_ctx* ctx);
int sps_launch_near_rev(sps_ctx* ctx);
int sps_launch_contacts(sps_ctx* ctx, int n, const double* pos, const double* radii);
// contacts, D products, identity-mobility BBPGD pieces (sps_contacts.cu)
int sps_check_inputs(sps_ctx* ctx, int n, const double* pos, const double* radii, const double* FT);
int sps_count_positive(sps_ctx* ctx, const double* v, int n, int* out);
// exclusive prefix sum of n ints on the context's stream (out may alias in)
int sps_exclusive_scan(sps_ctx* ctx, const int* in, int* out, long long n);
// the five BBPGD statistics land in sps_bb_out(ctx) (device, 5 doubles)
int sps_bb_stats_dev(sps_ctx* ctx, const double* gn, const double* ggn, const double* go,
                     const double* ggo);
int sps_launch_bb_identity(sps_ctx* ctx, double alpha, const double* gam, const double* g,
                           double* gam_new, double* g_new);
const double* sps_bb_out(sps_ctx* ctx);
int sps_launch_identity_U(sps_ctx* ctx, int n, const double* FT, const double* F3, double* UO);
int sps_launch_contact_grad(sps_ctx* ctx, const double* pos, const double* mu, const double* w,
                            const double* U, double dt, double* dx);
int sps_launch_D(sps_ctx* ctx, const double* gamma, double* FT);
int sps_launch_DT(sps_ctx* ctx, const double* UO, double* out);
int sps_launch_rho(sps_ctx* ctx, const double* FT, double* rho);
int sps_launch_moments(sps_ctx* ctx, const double* f, double* mom);
int sps_launch_add_L(sps_ctx* ctx, const double* mom, double* out);
int sps_launch_extract(sps_ctx* ctx, const double* mom, double* UO);

// layer operators (sps_vsh.cu, sps_nbody.cu)
int sps_launch_analysis(sps_ctx* ctx, const double* sig, bool fp32);
// tensor-core transforms (sps_sht_tc.cu)
int sps_sht_tc_upload(sps_ctx* ctx, sps_ctx::TcMat& out, const std::vector<double>& M, int R, int C);
int sps_launch_sht_tc(sps_ctx* ctx, const sps_ctx::TcMat& m, int mode, const double* in, double* out,
                      int scale_by_radius, const double* sig, int half);
int sps_sht_tc_status(sps_ctx* ctx);
int sps_launch_self(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32);
int sps_launch_near(sps_ctx* ctx, int op, double* out, bool fp32);
int sps_launch_far(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32);
int sps_launch_far_T32(sps_ctx* ctx, int op, const double* v, double* out);
int sps_layer(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32);

// generic batched product (sps_vsh.cu): mode 0 in = planes, out = rows (N x R);
// mode 1 in = rows (N x C), out = planes; FP64
int sps_launch_batched(sps_ctx* ctx, int mode, const double* M, int R, int C, const double* in, double* out,
                       int scale_by_radius, const double* sig, int half);
// adjoint helpers (sps_geometry.cu, sps_adjoint.cu)
int sps_launch_moments_w(sps_ctx* ctx, const double* f, double* mom, bool weighted);
int sps_launch_add_L_w(sps_ctx* ctx, const double* mom, double* out, bool weight_out);
int sps_layer_T(sps_ctx* ctx, int op, const double* v, double* out);

// near-field coefficient maps (sps_vsh.cu)
int sps_build_field_maps(sps_ctx* ctx);
// out32 / outdw (optional): copies of the result rounded to FP32 / split
// into FP32 hi + lo pairs (not with accumulate)
int sps_launch_sparse_rows(sps_ctx* ctx, const sps_ctx::Sparse& m, int nsph, const double* in, int in_ld,
                           double* out, int out_ld, int accumulate, float* out32 = nullptr,
                           float2* outdw = nullptr);

// vector kernels (sps_solver.cu)
int sps_dot(sps_ctx* ctx, const double* a, const double* b, long long n, double* host_out);
