// Internal scene state and host-side launchers of the HOT library.
#pragma once

#include "common.cuh"

namespace hot {

constexpr int MAX_LEVELS = 8;
constexpr int MAX_HIST = 16;
constexpr int DEVICE_LOOP_MIN_ITERS = 8;
// warps (rows) per block of the one-launch-per-color sweeps, from options flag bits 8-9
inline int sgs_color_warps(int flags) {
  static const int w[4] = {8, 2, 4, 16};
  return w[(flags >> 8) & 3];
}
constexpr int NSLOT = 125;       // 5^3 block offsets per row (Sec. 6 "Sparse matrix storage")
constexpr int DIAG_SLOT = 62;    // offset (0,0,0)

// particle field offsets in the SoA double array (field f of particle p at pd[f*np + p])
enum : int { PF_X = 0, PF_V = 3, PF_C = 6, PF_F = 15, PF_VOL = 24, PF_MASS = 25, PF_COUNT = 26 };

struct StencilGeom {
  int dims[3];        // cells per axis
  double dx, inv_dx;
  double origin[3];
  int nb[3];          // 4^3-cell blocks per axis
};

// precision-independent topology of one multigrid level
struct Topo {
  int64_t n = 0;      // active nodes
  int64_t nnzb = 0;   // 3x3 blocks
  int dims[3] = {0, 0, 0};   // dense node map extent (nodes per axis)
  DBuf<uint8_t> flag;        // dense activity flags
  DBuf<int> map;             // dense node -> compact index, -1 inactive
  DBuf<int> coords;          // 3n node triples
  DBuf<int> row_ptr;         // n+1
  DBuf<int> cols;            // nnzb
  DBuf<int> slotpos;         // 125 n: block position of (row, offset slot), -1 absent
  DBuf<uint32_t> mask;       // 4 n: present offset slots
  DBuf<int> rowcnt;          // n
  DBuf<int> nlow;            // n: blocks of neighbours colored before the row (a prefix of the row)
  DBuf<int> color_list;      // n, grouped by color
  DBuf<int> color_cnt;       // 28
  DBuf<int4> color_rec;      // n, (row, row_ptr[row], blocks in row, nlow[row]) in color_list order
  int color_off[28] = {0};   // host copy of the per-color offsets
  void set_stream(cudaStream_t st) {
    flag.st = st; map.st = coords.st = row_ptr.st = cols.st = slotpos.st = rowcnt.st = nlow.st = st;
    mask.st = st; color_list.st = color_cnt.st = st; color_rec.st = st;
  }
  size_t bytes() const {
    return flag.bytes() + map.bytes() + coords.bytes() + row_ptr.bytes() + cols.bytes() +
           slotpos.bytes() + mask.bytes() + rowcnt.bytes() + nlow.bytes() + color_list.bytes() + color_cnt.bytes() +
           color_rec.bytes();
  }
  void release() {
    flag.release(); map.release(); coords.release(); row_ptr.release(); cols.release();
    slotpos.release(); mask.release(); rowcnt.release(); nlow.release(); color_list.release(); color_cnt.release();
    color_rec.release();
  }
};

// values of one level in the hierarchy's precision
template <class T>
struct Vals {
  DBuf<T> vals;              // 9 nnzb; row i keeps entry e of its b-th block at 9*row_ptr[i] + e*nb_i + b
  DBuf<T> dinv;              // 9 n inverse diagonal blocks
  DBuf<T> diag;              // 3 n scalar diagonal
  DBuf<T> u, b, r;           // 3n level vectors
  void set_stream(cudaStream_t st) { vals.st = dinv.st = diag.st = u.st = b.st = r.st = st; }
  size_t bytes() const {
    return vals.bytes() + dinv.bytes() + diag.bytes() + u.bytes() + b.bytes() + r.bytes();
  }
  void release() { vals.release(); dinv.release(); diag.release(); u.release(); b.release(); r.release(); }
};

template <class T>
struct Hier {
  Vals<T> L[MAX_LEVELS];
  DBuf<T> A45;                         // per-particle projected stiffness
  DBuf<T> rap_t;                       // Galerkin product, first factor: H R^T per fine row (576 values)
  DBuf<T> x, r, z, p, Ap;              // coarsest PCG vectors
  DBuf<double> part;                   // PCG partial sums
  DBuf<unsigned int> bar;              // grid barrier words
  DBuf<int> cg_log;                    // PCG iteration counts; last entry = count
  int cl_level = -1;                   // coarsest level planned for the cluster solver (-1: none)
  int cl_size = 0;                     // CTAs in the cluster (16 or 8)
  int cl_bounds[17] = {0};
  int cl_rows_max = 0, cl_nb_max = 0;
  size_t cl_smem = 0;                  // 0: level does not fit one cluster
  void set_stream(cudaStream_t st) {
    for (auto &l : L) l.set_stream(st);
    A45.st = x.st = r.st = z.st = p.st = Ap.st = rap_t.st = st;
    part.st = st;
    bar.st = st;
    cg_log.st = st;
  }
  size_t bytes() const {
    size_t b = A45.bytes() + rap_t.bytes() + x.bytes() + r.bytes() + z.bytes() + p.bytes() + Ap.bytes() +
               part.bytes() + bar.bytes() + cg_log.bytes();
    for (auto &l : L) b += l.bytes();
    return b;
  }
  void release() {
    for (auto &l : L) l.release();
    A45.release(); rap_t.release(); x.release(); r.release(); z.release(); p.release(); Ap.release();
    part.release(); bar.release(); cg_log.release();
  }
};

enum Phase { PH_IDLE = 0, PH_P2G = 1, PH_HIER = 2, PH_SOLVED = 3 };

struct Trace {
  int iters = 0;
  std::vector<double> alphas;
  std::vector<int> ls_trials, skipped, fallback, cg_counts;
  std::vector<int> inner;   // CG iterations per Newton iteration (projected-Newton solvers)
  void clear() {
    iters = 0;
    alphas.clear(); ls_trials.clear(); skipped.clear(); fallback.clear(); cg_counts.clear(); inner.clear();
  }
};

// Scalars of the projected-Newton CG loop, in device memory.
struct CgState {
  double rz, bn, k, pAp, alpha, beta;
  int it, stop;
};

// The captured CG loop of the projected-Newton solvers (one per solve).
struct PnGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long top_kernels = 0, body_kernels = 0, upd_kernels = 0;
};

// Scalars of the device-driven L-BFGS loop (Alg. 3), in device memory.
struct LoopState {
  double E, E1, alpha, pg, n0, n1, nrm;
  double rho[MAX_HIST];
  int it, t, ok, fb, hist_n, head, status, trials_total;
};

struct Scene;
// Opt-in device timing of one kernel launch (CUDA events on the scene's
// stream around the launch); no cost when the scene's profiling is off.
struct ProfScope {
  Scene *s;
  int id;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(Scene &sc, const char *name);
  ~ProfScope();
};

struct Scene {
  // configuration
  int64_t np = 0;
  StencilGeom geo;
  double gravity[3];
  std::vector<mpm_material> mats;
  std::vector<mpm_bc> bcs;
  mpm_solver_opts opts;
  cudaStream_t st = nullptr;
  int nsm = 152;
  std::string last_error;
  Phase phase = PH_IDLE;
  bool has_grid = false;       // a P2G has run; its grid stays readable until the next one
  bool has_solution = false;   // dv holds the last solve of that grid
  double dt = 0.0;
  long long spin_limit = 1ll << 24;   // polls before a device-side wait gives up (mpm_set_wait_limit)

  // particles (sorted by cell after P2G); pd: PF_COUNT fields, SoA
  DBuf<double> pd, pd_alt;
  DBuf<int> pmat, pmat_alt, pid, pid_alt;
  DBuf<MatParams> mat_table;
  DBuf<mpm_bc> bc_dev;
  DBuf<unsigned int> key;      // block-major cell key per particle
  DBuf<int> slot, perm, tmp;
  // cells
  int64_t ncell_dense = 0;
  DBuf<int> cell_count, cell_start;
  int64_t n_cells = 0, n_blocks = 0;
  DBuf<int> cell_first, cell_n, cell_key;   // occupied cells
  DBuf<int> blk_first, blk_end, blk_key;    // occupied 4^3-cell blocks
  DBuf<int> flags;                          // per-particle segment flags / offsets
  DBuf<int> flag_scan;

  // grid level 0 (node data)
  DBuf<double> m, v, xi;       // n, 3n, n
  DBuf<uint8_t> fixed;         // n
  DBuf<double> mv, mxi;        // P2G accumulators

  // solver vectors (3n doubles)
  DBuf<double> dv, g, pdir, q, g_new, dv_new, vtmp;
  DBuf<double> hist_s, hist_y; // MAX_HIST x 3n
  DBuf<double> Lv, Lp;         // 9 np: sum_i u_i grad w_ip^T for v^n+dv and for p
  DBuf<double> Le, dv_e, g_e;  // scratch of the evaluation entry points
  DBuf<double> gscr;           // 54 np: per-particle factor tables of the gradient
  DBuf<double> part;           // partial sums
  DBuf<double> scal;           // device scalars
  DBuf<int> errflag;
  ScanScratch scan;
  DBuf<LoopState> lstate;      // device-driven loop scalars
  DBuf<double> cg_r, cg_z, cg_p, cg_Ap;   // projected-Newton CG vectors (3n)
  DBuf<CgState> cgs;
  PnGraph pn_graph;
  DBuf<double> tr_alpha;       // device-driven loop trace: step lengths
  DBuf<int> tr_int;            // ... line-search trials | skipped pairs | fallbacks
  cudaStream_t aux_st[2] = {nullptr, nullptr};   // streams for captures of conditional bodies
  bool loop_graph_ok = true;
  int last_iters = -1;             // L-BFGS iterations of the previous solve
  double last_step_s = 0.0;        // host time of the scene's last step in mpm_step_batch

  // parked: every device buffer released, the particle state (sorted SoA,
  // material ids, original ids) kept in host memory (mpm_scene_park)
  bool parked = false;
  std::vector<double> host_pd;
  std::vector<int> host_pmat, host_pid;
  size_t peak_bytes = 0;       // largest device footprint seen (admission estimate while parked)

  int nlev = 0;
  Topo topo[MAX_LEVELS];
  Hier<double> hd;
  Hier<float> hf;

  // L-BFGS bookkeeping (host)
  int hist_n = 0, hist_head = 0;
  double hist_rho[MAX_HIST];

  Trace trace;
  mpm_step_stats last_stats;

  // the V-cycle as a CUDA graph (re-captured whenever the hierarchy changes)
  bool graphs_ok = true;
  int graph_launches = 0;
  bool own_stream = false;
  cudaGraphExec_t vgraph = nullptr;
  const void *vgraph_b = nullptr, *vgraph_u = nullptr;
  long long vgraph_kernels = 0;   // kernels in the captured V-cycle
  void drop_graph() {
    if (vgraph) cudaGraphExecDestroy(vgraph);
    vgraph = nullptr;
  }

  // per-kernel device timing
  bool prof = false;
  std::string prof_only;                // record only these kernel names (comma-separated) when non-empty
  std::vector<std::string> prof_names;
  std::vector<int> prof_ids;
  std::vector<cudaEvent_t> prof_ev;     // start/stop pairs, in launch order
  std::vector<cudaEvent_t> ev_pool;

  int64_t nn() const { return topo[0].n; }
  void set_stream(cudaStream_t s) {
    st = s;
    for (auto *b : {&pd, &pd_alt, &m, &v, &xi, &mv, &mxi, &dv, &g, &pdir, &q, &g_new, &dv_new, &vtmp,
                    &hist_s, &hist_y, &Lv, &Lp, &part, &scal, &Le, &dv_e, &g_e, &gscr, &tr_alpha})
      b->st = s;
    for (auto *b : {&pmat, &pmat_alt, &pid, &pid_alt, &slot, &perm, &tmp, &cell_count, &cell_start,
                    &cell_first, &cell_n, &cell_key, &blk_first, &blk_end, &blk_key, &flags, &flag_scan,
                    &errflag, &tr_int})
      b->st = s;
    key.st = s;
    fixed.st = s;
    lstate.st = s;
    cgs.st = s;
    cg_r.st = cg_z.st = cg_p.st = cg_Ap.st = s;
    mat_table.st = s;
    bc_dev.st = s;
    scan.block_sums.st = scan.total.st = s;
    for (auto &t : topo) t.set_stream(s);
    hd.set_stream(s);
    hf.set_stream(s);
  }
  size_t bytes() const;
  void release();
};

// ---- transfer.cu
void compact_dense(Scene &s, Topo &T);   // dense flags -> map, coords, n
void bin_and_sort(Scene &s);
void build_level0_nodes(Scene &s);
void p2g_transfer(Scene &s);
double max_particle_speed(Scene &s);
void g2p_transfer(Scene &s, const double *vnew);
void scatter_state_to_user_order(Scene &s, double *x, double *v, double *F, double *C, bool to_device);
void load_state_from_user_order(Scene &s, const double *x, const double *v, const double *F,
                                const double *C, bool from_device);

// ---- elastic.cu
// L_p = sum_i (u_i [+ u2_i]) grad w_ip^T per particle (u2 may be NULL)
void velocity_gradient(Scene &s, const double *u, const double *u2, double *L);
// E(dv + alpha p): particles use F = (I + dt (L1 + alpha L2)) F^n, nodes use
// dv + alpha p (L2 and p may be NULL when alpha = 0)
double energy(Scene &s, const double *L1, const double *L2, double alpha, const double *dv, const double *p);
// launch only: partials of the energy into s.part (returns their count); the
// step length is read from alpha_dev when it is not NULL
int energy_launch(Scene &s, const double *L1, const double *L2, double alpha, const double *alpha_dev,
                  const double *dv, const double *p);
// gradient at the state whose velocity gradient is L and node increment dvec;
// norms_out[0] = ||g||^2, norms_out[1] = ||g^||^2 (CN-scaled), both host
void gradient(Scene &s, const double *L, const double *dvec, double *gout, double norms_out[2]);
// launch only: gradient into gout, norm partials (pairs) into s.part; returns the pair count
int gradient_launch(Scene &s, const double *L, const double *dvec, double *gout);
template <class T>
void particle_stiffness(Scene &s, Hier<T> &h);
template <class T>
void hessian_assemble(Scene &s, Hier<T> &h);

// ---- multigrid.cu
void build_pattern0(Scene &s);
void build_coarse_topology(Scene &s, int m);   // level m+1 nodes and pattern from level m
void build_colors(Scene &s, int m);
template <class T>
void rap(Scene &s, Hier<T> &h, int m);          // numeric H^{m+1} = R H^m R^T
template <class T>
void finalize_values(Scene &s, Hier<T> &h, int m);   // diagonal inverses
// Alg. 2 on b_in (3n doubles, level 0) -> u_out, asynchronous; the coarsest
// PCG appends its iteration count to a device log
template <class T>
void vcycle(Scene &s, Hier<T> &h, const double *b_in, double *u_out, bool use_graph);
template <class T>
void vcycle_ready(Scene &s, Hier<T> &h);                                      // before a capture
template <class T>
void vcycle_emit(Scene &s, Hier<T> &h, const double *b_in, double *u_out);   // launches only
template <class T>
void reset_cg_log(Scene &s, Hier<T> &h);
template <class T>
std::vector<int> read_cg_log(Scene &s, Hier<T> &h);

// ---- vecops.cu (deterministic: fixed grid, fixed-order partial sums)
double dot(Scene &s, const double *x, const double *y, int64_t n);
// out = {x.y, x.x, y.y}
void dots3(Scene &s, const double *x, const double *y, int64_t n, double out[3]);
void axpy(Scene &s, double *y, double a, const double *x, int64_t n);                 // y += a x
void lincomb(Scene &s, double *z, double a, const double *x, double b, const double *y, int64_t n);  // z = a x + b y
void scale_copy(Scene &s, double *dst, double a, const double *src, int64_t n);       // dst = a src
int64_t count_free(Scene &s);                                                         // nodes with fixed == 0
// L-BFGS two-loop recursion of Alg. 3 around the initial inverse, with the
// step scalars kept on the device.  First half turns q into the V-cycle
// input; second half turns r (the V-cycle output) into the direction.
void two_loop_first(Scene &s, double *q, int64_t n);
void two_loop_second(Scene &s, double *r, int64_t n);
// The same with the pair count, history head and rho read from a LoopState
// on the device (a fixed launch sequence, inactive steps do nothing).
void two_loop_first_dev(Scene &s, double *q, int64_t n, const LoopState *st);
void two_loop_second_dev(Scene &s, double *r, int64_t n, const LoopState *st);
// launch only: k_dot3 partials (triples, one per block) into part; returns the block count
int dot_launch(Scene &s, const double *x, const double *y, int64_t n, int mode, double *part);
// {y.s, y.y, s.s} partials of the history pair in slot st->head
int dots3_hist_launch(Scene &s, int64_t n, const LoopState *st, double *part);
void lincomb_alpha(Scene &s, double *z, const double *x, const double *y, int64_t n, const LoopState *st);  // z = x + alpha y
void axpy_alpha(Scene &s, double *y, const double *x, int64_t n, const LoopState *st);                     // y += alpha x
void hist_diff(Scene &s, double *base, const double *x, const double *y, int64_t n, const LoopState *st);  // slot head of base = x - y

// ---- solve_graph.cu
// Alg. 3's iterations as one CUDA graph with conditional nodes (device-side
// decisions); returns false, touching nothing, when the graph cannot be built.
bool solve_loop_graph(Scene &s, double E0, double norms0[2], double thr, double &E, double &nrm, int &it,
                      int &trials_total, mpm_status &status);

// ---- newton.cu (Alg. 1, the comparison solvers)
void pn_prepare(Scene &s);          // captures the CG loop (buffers, V-cycle plan first)
int pn_cg_run(Scene &s);            // CG on H p = -g into s.pdir; returns its iterations
void pn_release(Scene &s);
void pn_rebuild_values(Scene &s);   // projected Hessian (and hierarchy) at the current s.Lv
                                    // (also the refresh extension of the L-BFGS loop)
void note_launches(long long n);   // adds to the kernel launch counter
long long launch_count();

int read_errflag(Scene &s);
bool prof_selected(const std::string &only, const char *name);   // api.cu: is `name` in the filter

// ---- api.cu: refresh rule of the hierarchy-refresh extension
bool refresh_due(const mpm_solver_opts &o, int it);

// ---- api.cu: residency
void park_scene(Scene &s);        // device buffers -> host copy of the particle state, buffers released
void ensure_resident(Scene &s);   // the reverse, when parked

}  // namespace hot
