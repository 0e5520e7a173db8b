// Internal description of one set-up system: sizes, device index tables and
// device buffers.  Shared by the host driver and the per-precision kernel units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace ltmp2 {

// Operands, tensor maps and error flag of the tcgen05 3xTF32 GEMM (precision form).
struct OzResources;   // FP64 tensor-core GEMM resources (below)
struct TcResources {
  int rows_cap = 0, npw = 0, kpad = 0;
  int variant = 5;         // 4 drained N=64, 5 stacked Re/Im rows (default; the only one for real orbitals)
  bool real = false;       // real-basis Green's function: K = n_pw (variant 5 only)
  float *a1h = nullptr, *a1l = nullptr, *a2h = nullptr, *a2l = nullptr, *bh = nullptr, *bl = nullptr;
  int *err = nullptr;      // device flag: a bounded wait ran out
  void *maps = nullptr;    // host copy of the six TMA tensor maps
  // Green's function on the tensor cores (real basis): P_r = R_v^T D R_v with K = n_v,
  // two real rows of R_v^T D per complex row of the stacked kernel
  bool green = false;
  int nv = 0, kpad_v = 0, grows = 0;   // virtuals, padded K, complex rows ceil(n_pw / 2)
  float *rvt = nullptr;                // [n_pw][n_v] R_v^T
  float *gah = nullptr, *gal = nullptr, *gbh = nullptr, *gbl = nullptr;
  void *gmaps = nullptr;               // host copy of the four tensor maps
  // direct term on the tensor cores (real basis): one product per primary G' of a slab
  bool direct = false;
  int dno = 0, dr64 = 0, dkpad = 0, dnaux = 0, dslots = 0;
  float *dah = nullptr, *dal = nullptr, *dbh = nullptr, *dbl = nullptr;
  float2 *dc = nullptr;                // [slots][n_o][2 n_o]
  void *dmaps = nullptr;
  // whether the set-up Green's function / direct-term products are used (ltmp2_set_tuning);
  // otherwise the CUDA-core kernels run
  bool use_green = false, use_direct = false;
  bool green_on() const { return green && use_green; }
  bool direct_on() const { return direct && use_direct; }
};
int tc_kpad(int npw);
size_t tc_bytes(int rows_cap, int npw);
cudaError_t tc_init(TcResources &r, void *mem, int rows_cap, int npw, int variant, bool real = false);
int tc_variant_bn(int variant);
void tc_release(TcResources &r);
cudaError_t tc_pack_b(const TcResources &r, const void *pt, cudaStream_t st);
// Green's function on the tensor cores: device bytes, set-up (transpose and split of the
// virtuals' real coordinates cv [n_v][n_pw], once) and one build into pt (pair-interleaved)
size_t tc_green_bytes(int npw, int nv);
cudaError_t tc_green_init(TcResources &r, void *mem, const float *cv, int nv, cudaStream_t st);
cudaError_t tc_green(const TcResources &r, const float *dv, void *pt, cudaStream_t st);
// direct term on the tensor cores: bytes and set-up for up to `slots` primary G' per slab,
// and the pair sums Y [np][n_o][n_o] of one slab from its diagonal co-densities
size_t tc_direct_bytes(int no, int naux, int slots);
cudaError_t tc_direct_init(TcResources &r, void *mem, int no, int naux, int slots);
cudaError_t tc_direct(const TcResources &r, const void *mdiag, const float *v, int np, double2 *yd, cudaStream_t st);
cudaError_t tc_wgemm(const TcResources &r, const void *st_in, int rows, void *wt, cudaStream_t st);
// one bounded wait on an mbarrier that never completes (failure-path self-test)
cudaError_t tc_wait_selftest(int *err, unsigned long long limit_ns, cudaStream_t st);

// One column of a plane-wave sphere at fixed (m1, m2): m3 runs over [zlo, zhi].
// Columns are stored in order; the sphere's points follow column by column
// (m3 ascending), starting at col_off[c].
struct Plan {
  int n = 0;                 // FFT grid points per axis (cubic grid)
  int n_occ = 0, n_orb = 0, n_pw = 0, n_v = 0;
  int n_dorb = 0;            // orbital-sphere columns
  int n_daux = 0;            // aux-sphere columns
  int n_aux = 0;             // |A|
  int n_prim = 0;            // primary G' (first non-zero Miller index > 0)
  int mxlo_orb = 0, mxhi_orb = 0, mxlo_aux = 0, mxhi_aux = 0;
  bool real_orb = false;
  // real_orb and the Green's function is built in the real cos/sin basis: cv holds the
  // real coordinates of the virtuals, pt the real symmetric P_v, and the W product is
  // complex x real (half the multiply-adds of the complex product)
  bool real_basis = false;
  int precision = 0;         // 0 = FP64, 1 = FP32
  double omega = 0.0, mu = 0.0;

  // device index tables
  int4 *dorb = nullptr;      // [n_dorb] (m1, m2, zlo, zhi)
  int *dorb_off = nullptr;   // [n_dorb]
  int4 *daux = nullptr;      // [n_daux]
  int *daux_off = nullptr;   // [n_daux]
  int *pw_m = nullptr;       // [n_pw * 3] Miller indices of the orbital sphere, internal order
  int *pw_pair = nullptr;    // [n_pw] internal position of -G_q (real basis only)
  int *aux_m = nullptr;      // [n_aux * 3]
  int *aux_neg = nullptr;    // [n_aux] position of -G in A
  int *prim = nullptr;       // [n_prim] position in A of each primary G'
  double *v_aux64 = nullptr; // [n_aux] 4 pi / |G|^2
  float *v_aux32 = nullptr;
  double *eps = nullptr;     // [n_orb] (device)

  // precision-dependent device data (cpx<T>)
  void *cv = nullptr;        // [n_v][n_pw] virtual coefficients, internal order (T if real_basis)
  void *cgrid = nullptr;     // [n_occ][n^3] occupied coefficients scattered on the grid
  void *u = nullptr;         // [n_occ][n^3] occupied orbitals in real space, [z][y][x]
  void *ut = nullptr;        // [n_occ][n^3] the same, each z plane transposed: [z][x][y]
  void *utr = nullptr;       // real orbitals at Gamma: the real part of ut, T [n_occ][z][x][y]
                             // (the orbitals are real in real space), else null
  void *dscale = nullptr;    // [n_orb] T: virtual e^{-(e_a-mu)tau}, occupied e^{(e_j-mu)tau}
  void *pt = nullptr;        // [n_pw][n_pw] transposed Green's function P^T (real P if real_basis)
  void *st = nullptr;        // [max_cols][n_pw] gathered, scaled e^{-iG'r}|j> (S^T)
  void *wt = nullptr;        // [max_cols][n_pw] transformed states W^T
  void *z1 = nullptr;        // [max_cols][n][n_dorb] W after the inverse z transform
  void *tbuf = nullptr;      // [max_cols * n_occ][n][n_daux] co-densities after the xy transform
  void *mdiag = nullptr;     // [max_slots][n_aux][n_occ] diagonal co-densities M_ii(G;G')
  double2 *sx = nullptr;     // [max_prim][n_occ][n_occ] exchange pair sums X_ij(G')
  double2 *yd = nullptr;     // [max_prim][n_occ][n_occ] direct pair sums Y_ij(G')
  double *ex = nullptr, *ed = nullptr, *exi = nullptr, *edi = nullptr;  // [n_occ][n_occ]
  double *esum = nullptr;    // [4]: E_d, E_x, imag parts
  int max_prim = 0;          // primary G' per slab (capacity)
  TcResources *tc = nullptr; // precision form: tcgen05 GEMM resources (host pointer), or null
  OzResources *oz = nullptr; // FP64 path: tensor-core FP64 GEMM resources (host pointer), or null
  int plane_kernel = 2;      // 0: k_planes, 1: k_planes2, 2: k_planes3, 3: k_planes4 (set-up: 3 in FP32;
                             // the autotuner may change it)
  // screened exchange pairs (learned form); all null = every pair contracted
  const unsigned char *pair_keep = nullptr;  // [n_occ][n_occ] 1 = contract, symmetric, diagonal kept
  const int *keep_list = nullptr;            // [n_occ][n_occ] kept i for each j (first keep_count[j])
  const int *keep_count = nullptr;           // [n_occ]
  int plane_ib = 0;          // occupied planes per plane-kernel block, 0 = kernel default
  // internal auxiliary-cutoff extrapolation (Sec. III D): nested spheres A_1 = A, ...,
  // A_n = {G : |G|^2/2 <= E_aux / alpha^(n-1)}; every G- and G'-sum is also kept per level.
  // n_lev < 2: off.
  int n_lev = 0;
  const unsigned char *aux_lev = nullptr;  // [n_aux] L(G): G belongs to A_1 .. A_L(G)
  const int *lev_order = nullptr;          // [n_aux] aux positions grouped by L (L = 1 first)
  const int *lev_start = nullptr;          // [n_lev + 1] group boundaries in lev_order
  size_t lev_stride = 0;                   // elements per level of sxl / ydl
  double2 *sxl = nullptr, *ydl = nullptr;  // [n_lev][slab cap][n_occ][n_occ] pair sums over A_n
  double *exl = nullptr, *edl = nullptr;   // [n_lev][n_occ][n_occ] level pair energies (n >= 2)
  double *esum_lev = nullptr;              // [2 n_lev]: E_d[n], E_x[n]
  // Transformed-state route.  0: Green's function P_v(tau) built per tau and applied to the
  // gathered e^{-iG'r}|j> (W = P_r (U S)).  1: the paper's route, Sec. III A steps (i)-(iii):
  // overlap densities rho_aj(G') = <a|e^{-iG'r}|j> stored once (rt), and per tau
  // W = sum_a |a> e^{-(e_a-mu)tau} rho_aj(G') e^{(e_j-mu)tau} (real orbitals only).
  int route = 0;
  void *rt = nullptr;        // route 1: [n_prim * n_occ][n_v] cpx<T>, row (G', j), column a
  // Virtuals that carry weight at the current tau.  Energies ascend, so the virtuals with
  // e^{-(e_a - e_LUMO) tau} >= 2^-L are the first nv_tau of them; the others are left out
  // of the Green's function and of the transformed states (0 = all n_v).  With w_virtual
  // the transformed states go through the virtual space, W^T = ((U S)^T R_v'^T D') R_v'
  // (real basis, CUDA-core GEMMs; rvt = R_v^T [n_pw][n_v]), which costs 4 n_pw nv_tau
  // multiply-adds per column against 2 n_pw^2 through P_r, and no Green's function is built.
  int nv_tau = 0;
  bool w_virtual = false;
  void *rvt = nullptr;
  // k-point sampling (Sec. II C-D), nk > 0: n_occ counts composite occupied orbitals
  // k n_o + i over the mesh, n_orb / n_v are per k, cv [nk][n_v][n_pw], pt [nk][n_pw][n_pw],
  // dscale [nk][n_orb]; the auxiliary set A (daux, aux_m) is the ball that holds every
  // momentum-transfer class; the outer loop runs over primary supercell transfers Q'.
  int nk = 0;
  int mesh[3] = {1, 1, 1};
  int no_k = 0;                        // occupied per k
  const int *prim_m = nullptr;         // [n_prim][3] supercell Miller index of each primary Q'
  const double *vprim = nullptr;       // [n_prim] 4 pi / |Q'|^2
  const double *vcls64 = nullptr;      // [n_cls][n_aux] 4 pi / |g + delta/n|^2 inside the sphere, else 0
  const float *vcls32 = nullptr;
  const int *lut = nullptr;            // [n^3] position in A of the grid point, -1 if absent
  int slots_per_prim() const { return (real_orb && nk == 0) ? 1 : 2; }
};

// FP64 products on the tensor cores by exact integer slices (gemm_f64tc.cuh): the FP64
// path's transformed-state GEMM in the real basis, W^T = (U S)^T P_r.
struct OzResources {
  int rows_cap = 0, npw = 0, kpad = 0, arows = 0;  // complex rows, K = n_pw, padded K, stacked rows
  int nv = 0;                                      // virtuals (rows of the static slices bv)
  float *a = nullptr, *b = nullptr;                // slices [8][arows][kpad], [8][npw][kpad]
  float *bv = nullptr;                             // slices of R_v [8][nv][kpad], once per context
  double *sa = nullptr, *sb = nullptr, *sbv = nullptr;  // row scales (powers of two)
  int *err = nullptr;                              // device flag: a bounded wait ran out
  void *maps = nullptr;                            // host copy of the three tensor maps
};
size_t oz_bytes(int rows_cap, int npw, int nv);
cudaError_t oz_init(OzResources &r, void *mem, int rows_cap, int npw, int nv);
void oz_release(OzResources &r);
// slices of the virtuals' real coordinates R_v (cv [nv][npw]), once
cudaError_t oz_split_cv(const OzResources &r, const double *cv, cudaStream_t st);
// the Green's function P_r = R_v'^T D' R_v' over the first nv virtuals (dv: their weights)
// into pr [npw][npw]; needs oz_green_fits (n_pw rows fit the A slices)
bool oz_green_fits(const OzResources &r);
cudaError_t oz_green(const OzResources &r, const double *rvt, const double *dv, int nv, double *pr, cudaStream_t st);
// W^T through the virtual space: X^T = S^T R_v'^T into x (complex [rows][nv]), then
// W^T = X^T D' R_v' into wt (complex [rows][npw])
cudaError_t oz_virtual(const OzResources &r, const void *st_in, int rows, const double *rvt, const double *dv, int nv,
                       void *x, void *wt, cudaStream_t st);
// slices of P_r (real symmetric [npw][npw]) as the B operand, once per tau
cudaError_t oz_split_b(const OzResources &r, const double *pr, cudaStream_t st);
// W^T (complex [rows][npw]) = S^T (complex [rows][npw]) P_r
cudaError_t oz_wgemm(const OzResources &r, const void *st_in, int rows, void *wt, cudaStream_t st);
// the bounded-wait flag: LTMP2_OK, or LTMP2_ERR_TIMEOUT (flag cleared), or LTMP2_ERR_CUDA
int oz_check(const OzResources &r);

// Per-stage profiler hooks (host).  begin/end bracket one kernel launch.
struct StageTimer {
  virtual void begin(int stage) = 0;
  virtual void end(int stage) = 0;
  virtual ~StageTimer() {}
};

constexpr int kMaxLevels = 16;   // nested cutoffs of the internal extrapolation

// One round of the batching form's persistent stages: the active systems, their item ranges
// (plane items: N planes x columns; column items: pairs) and their slab.
constexpr int kBatchMax = 16;
constexpr int kPersistThreads = 128;
struct BatchRound {
  int nsys = 0;
  int first[kBatchMax + 1] = {0};   // item prefix over the active systems
  int sys[kBatchMax] = {0};         // index of each active system in the plan array
  int gp0[kBatchMax] = {0}, np[kBatchMax] = {0}, ib[kBatchMax] = {0};
};

enum Stage {
  kStageGreen = 0, kStageWGemm = 1, kStageGatherZ = 2, kStagePlane = 3,
  kStageColumn = 4, kStageDirect = 5, kStageAccum = 6
};

// Per-precision entry points (kernels_f64.cu / kernels_f32.cu)
template <typename T> struct Path {
  // kernel launches per Green's function build and per slab (the tcgen05 path of the
  // precision form adds one operand-packing launch to each)
  static int green_launches(const Plan &p) {
    if (p.route == 1 || p.w_virtual) return 1;
    if (p.tc) return p.tc->green_on() ? 4 : 3;
    if (p.oz) return oz_green_fits(*p.oz) && p.rvt ? 5 : 3;   // dscale, [split, split, product | product], split of P_r
    return 2;
  }
  static int slab_launches(const Plan &p) {
    if (p.route == 1) return 7 + (p.n_lev > 1 ? 1 : 0);   // no gather, CUDA-core product
    // W: one product; FP64 on the tensor cores: split + product; through the virtual space:
    // two products (CUDA cores) or split, product, split, split, product (tensor cores)
    const int w = p.w_virtual ? (p.oz ? 5 : 2) : (p.oz ? 2 : 1);
    return (p.tc ? 8 : 7) - 1 + w + (p.real_basis ? 1 : 0) + (p.n_lev > 1 ? 1 : 0) +
           (p.tc && p.tc->direct_on() && p.n_lev < 2 ? 2 : 0);   // direct term: pack, product, combine
  }
  // route 1 setup: the overlap densities of every primary G' into rt (uses st and pt as
  // scratch; pt holds the transposed virtual coordinates meanwhile)
  static cudaError_t overlap_setup(const Plan &p, cudaStream_t st);
  // launches of zero_acc + finish
  static int frame_launches(const Plan &p) { return p.n_lev > 1 ? 3 : 2; }
  static cudaError_t init_device();
  // setup: occupied orbitals -> u (real space) and cgrid
  static cudaError_t setup_occupied(const Plan &p, const void *c_occ_dev, cudaStream_t st);
  // one tau: scale factors and Green's function P^T
  static cudaError_t green(const Plan &p, double tau, cudaStream_t st, StageTimer *tm);
  // one slab of primary G' [gp0, gp0 + np): everything up to the pair sums, then accumulate
  static cudaError_t slab(const Plan &p, int gp0, int np, double coef, cudaStream_t st,
                          StageTimer *tm);
  // the slab in phases: up to w in real space (gather, transformed-state GEMM, z transform),
  // and after the co-density FFTs (direct term, accumulation); the batching form runs the
  // FFT stages of every system in between as shared persistent launches
  static cudaError_t slab_pre(const Plan &p, int gp0, int np, cudaStream_t st, StageTimer *tm);
  static cudaError_t slab_post(const Plan &p, int gp0, int np, double coef, cudaStream_t st, StageTimer *tm);
  // persistent plane / column kernels over the items of several systems (device plan array)
  static cudaError_t planes_persist(const Plan *d_plans, const struct BatchRound &r, int *counter, int blocks,
                                    size_t smem, cudaStream_t st);
  static cudaError_t zcol_persist(const Plan *d_plans, const struct BatchRound &r, int *counter, int blocks,
                                  size_t smem, cudaStream_t st);
  static size_t plane_smem_for(const Plan &p, int ib);
  static cudaError_t persist_attributes(size_t plane_smem, size_t col_smem);
  static int persist_blocks(bool planes, size_t smem);
  // plane kernel `kernel` with `ib` occupied planes per block fits the launch limits
  static bool plane_feasible(const Plan &p, int kernel, int ib);
  // the plane kernel alone (for the autotuner): kernel 0/1/2, ib (0 = default)
  static cudaError_t plane_pass(const Plan &p, int ncols, int kernel, int ib, cudaStream_t st);
  // per-orbital density moments [n_occ][6] and pair density overlaps [n_occ][n_occ] (device)
  static cudaError_t descriptors(const Plan &p, double *moments, double *overlap, cudaStream_t st);
  // k-point sampling: scale factors and the Green's function of every k for one tau, and
  // one slab of primary supercell transfers Q' [gp0, gp0 + np)
  static cudaError_t green_k(const Plan &p, double tau, cudaStream_t st, StageTimer *tm);
  static cudaError_t slab_k(const Plan &p, int gp0, int np, double coef, cudaStream_t st, StageTimer *tm);
  static int green_k_launches(const Plan &p) { return 1 + p.nk; }
  static int slab_k_launches(const Plan &p) { return 6 + p.nk; }
  // opposite-spin direct term of one slab (alpha plan pa, beta plan pb, same slab):
  // y [slab][na][nb] scratch, acc [na][nb] accumulated
  static cudaError_t direct_cross(const Plan &pa, const Plan &pb, int gp0, int np, double coef, double *y,
                                  double *acc, cudaStream_t st);
  static cudaError_t sum(int n, const double *x, double *out, cudaStream_t st);
  // zero accumulators / final reduction
  static cudaError_t zero_acc(const Plan &p, cudaStream_t st);
  static cudaError_t finish(const Plan &p, cudaStream_t st, StageTimer *tm);
};

}  // namespace ltmp2
