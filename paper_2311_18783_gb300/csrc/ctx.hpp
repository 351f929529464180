// The library context: host topology plus every device array of one problem.
#pragma once
#include "common.cuh"
#include "dense.cuh"
#include "topology.hpp"
#include "xi.hpp"

#include <memory>

namespace geneo {
struct Multifrontal;
struct MfDeleter {
  void operator()(Multifrontal *m) const;
};
struct TcFactors;
struct TcDeleter {
  void operator()(TcFactors *t) const;
};
struct Mlp;
}  // namespace geneo

// public handle of a warm-start network
struct geneo_mlp {
  geneo::Mlp *m = nullptr;
};

namespace geneo {
// one autotuned SYMV target: candidate timings and the configuration kept
struct TuneRecord {
  std::string target, key;
  int precision = 0, chosen = 0;
  bool from_cache = false;
  std::vector<double> ms;  // per candidate (empty when taken from the cache)
};
}  // namespace geneo

struct geneo_ctx {
  // problem copy
  int nx = 0, ny = 0, nz = 0;
  double h[3] = {0, 0, 0};
  double gamma = 0, tau = 0, tau_p = 0;
  int px = 0, py = 0, pz = 0, overlap = 0;
  std::vector<uint8_t> active;
  std::vector<double> mu_inv, eps;
  std::vector<int32_t> cell_part;  // explicit partition, empty for boxes
  std::vector<uint8_t> natural;    // natural boundary faces per cell, empty for none
  bool host_only = false;          // geneo_setup_topology: integer data only, no device
  // independent components (vertex-connected active cells): unknown ranges
  // [seg_off[s], seg_off[s+1]) when contiguous (seg_ok), per-unknown component
  std::vector<int64_t> seg_off;
  std::vector<int32_t> seg_of;  // component of every unknown
  bool seg_ok = false;
  geneo::DevBuf<int32_t> d_seg_of;
  geneo::DevBuf<int64_t> d_seg_off;
  geneo::DevBuf<double> seg_sc;     // per-component PCG scalars
  geneo::DevBuf<int> seg_act;
  std::vector<int> seg_ha;
  double *h_seg = nullptr;            // pinned host mirror of the per-component scalars
  cudaGraphExec_t seg_exec = nullptr; // CUDA graph of one segmented PCG iteration
  int seg_key = -1;
  int64_t seg_graph_launches = 0;
  geneo_options opt{};
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;  // internal set-up stream
  double setup_seconds = 0;
  // wall seconds of the set-up stages: assembly, local inverses, split /
  // bfloat16 factors, GenEO eigensolves, GenEO independence filter, coarse
  // factor, autotuning, total
  double stage_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<geneo::TuneRecord> tune;

  geneo::Topology topo;
  geneo::Decomposition dec;
  geneo::LocalStructure ls;
  geneo::SNKColumns snk;

  // mesh and global matrix
  geneo::DevBuf<int32_t> d_tets, d_tet_cell, d_tet_edges, d_edge_tail, d_edge_dir;
  geneo::DevBuf<double> d_mu, d_eps;
  geneo::DevBuf<double> d_Ae;                 // [ntets][36] element A_T
  geneo::DevBuf<int32_t> d_rowptr, d_col;
  geneo::DevBuf<double> d_val;
  // sliced ELLPACK copy of A (SpMV): slice offsets and widths, column
  // indices, values, sorted-position -> row
  int64_t sell_nslices = 0, sell_stored = 0;
  geneo::DevBuf<int64_t> d_sell_off;
  geneo::DevBuf<int32_t> d_sell_w, d_sell_col, d_sell_perm;
  geneo::DevBuf<double> d_sell_val;
  geneo::DevBuf<int64_t> d_cptr, d_rptr;
  geneo::DevBuf<int32_t> d_cidx, d_ridx;

  // local factors (tile-packed inverses of A_i)
  geneo::TileBatch loc;
  geneo::DevBuf<double> loc_f64;
  geneo::DevBuf<float> loc_f32;
  geneo::DevBuf<int32_t> d_l2g;               // [loc.vlen] unknown or -1
  geneo::DevBuf<int64_t> d_g2l_ptr, d_g2l;    // prolongation lists (padded slots)

  // coarse space: Z in CSC and CSR, dense E^-1 (tile-packed single matrix)
  int64_t n0 = 0, n0_snk = 0, n0_geneo = 0;
  std::vector<int32_t> geneo_sub, geneo_found;
  std::vector<double> geneo_lambda;
  std::vector<int64_t> zc_ptr;
  std::vector<int32_t> zc_row;
  std::vector<double> zc_val;
  geneo::DevBuf<int64_t> d_zc_ptr, d_zr_ptr;
  geneo::DevBuf<int32_t> d_zc_row, d_zr_col;
  geneo::DevBuf<double> d_zc_val, d_zr_val;
  geneo::TileBatch crs;
  geneo::DevBuf<double> crs_f64;

  // sparse coarse factor (multifrontal); the dense E^-1 above is the alternative
  std::unique_ptr<geneo::Multifrontal, geneo::MfDeleter> mf;

  // local operators (xi, S_j^-1, element data) for GenEO and the split solve
  std::unique_ptr<geneo::XiOp> xi;
  int local_prec = GENEO_PREC_FP64;  // precision used by the local solves
  bool balanced = false;             // PCG in the balanced (one coarse solve) form
  bool grad32 = false;               // split local solves: S_j^-1 in float32
  bool mf_persist = false;           // coarse solve as one cooperative launch
  // warm start of the local eigensolves: edge features [loc.vlen][5]; the
  // locked eigenvectors (first 8 per subdomain, and B times them) when kept
  geneo::DevBuf<float> d_feat;
  geneo::DevBuf<double> eigV, eigBV;
  std::vector<int32_t> eig_nq, lobpcg_iters, lobpcg_iters0;  // iterations: all rounds, first round
  // bfloat16 super-tiles of C_j for the tensor-core local solves
  std::unique_ptr<geneo::TcFactors, geneo::TcDeleter> tc;

  // work vectors
  geneo::DevBuf<double> v_y0, v_s, v_w, v_t, v_c, loc_x, loc_y, loc_xp, crs_x, crs_y;
  geneo::DevBuf<double> p_r, p_z, p_p, p_q, scal, partials;
  geneo::DevBuf<double> h_b, h_x;  // device copies used by geneo_solve_host
  geneo::DevBuf<double> ref_r, ref_d;  // refinement: accurate residual and correction
  geneo::DevBuf<double> gm_V, gm_Z;    // GMRES: Krylov basis and preconditioned basis
  int gm_cap = 0;
  geneo::DevBuf<int> d_err;
  double *h_scal = nullptr;  // pinned host mirror of the PCG scalars

  // profiling: host launch counter and event pairs around SYMV launches
  bool prof = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_local, ev_coarse;
  cudaEvent_t ev_take();
  // totals harvested from graph replays (the graph owns its event pairs)
  double acc_local_ms = 0, acc_coarse_ms = 0;
  int64_t acc_local_n = 0, acc_coarse_n = 0;

  // CUDA graph of one PCG iteration (preconditioner, p update, A p, x/r
  // update, dots, scalar read-back), rebuilt when the local precision or the
  // profiling switch changes
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  int pcg_key = -1;
  int64_t pcg_graph_launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_ev_local, g_ev_coarse;
  geneo::DevBuf<double> p_x;
  void drop_graph();

  // right-hand-side columns the work buffers hold; PCG column mask
  int kcap = 0;
  geneo::DevBuf<int> d_act;
  int *h_act = nullptr;

  ~geneo_ctx();
};
