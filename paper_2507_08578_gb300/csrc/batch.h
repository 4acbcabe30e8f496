// Batched lockstep engine shared by kss_solve_batch (batch.cu) and the request server (server.cu).
#pragma once

#include <vector>

#include "fft_reg.cuh"
#include "kss_internal.h"

namespace kss {

struct RegPlanHost {  // host copy of the per-unit FFT split plan (same layout as the device one)
  fftr::Split s1, s2, s3;
};
struct WsOff {
  size_t cprj, part, slab;
};
struct PassClass {  // units whose FFT passes share one kernel instance
  int code1, code23;  // compile-time split codes (A*32+B) or -1 for the runtime-sized form
  int first, count;   // range in the class-ordered item table
  int blocks_ac, blocks_b;
  size_t smem_ac, smem_b;
  size_t smem_bw;  // shared memory of the CTA-wide pass B form
  int wa, wb, wnt; // pass B schedule (autotuner): CTA-wide split wa x wb at wnt threads; wnt == 0:
                   // the per-warp form (split code code23)
  int fcode = 0;   // single precision, small cubic box: the fused single-kernel instance (split code
                   // A*32+B) runs the whole local part of the class in one persistent launch
  int ftasks = 0;  // its (unit, band) tasks
  size_t smem_f = 0;
};
struct Roles {
  int y, hy, free2;  // buffers holding Y, H Y, and the free one that receives the rotated X
};

class BatchEngine {
 public:
  kss_ctx ctx = nullptr;
  bool f64 = true;
  int degree = 10;
  bool use_graph = true;
  bool use_batched_rr = true;
  bool use_tc_gemm = true;  // single precision: projector products on the tensor cores

  ~BatchEngine();
  // One lockstep iteration over every unit of `all` that is not done (fresh units get their
  // initial Rayleigh-Ritz; the others one filter + Rayleigh-Ritz); one host synchronisation.
  void iterate(std::vector<kss_solver_s*>& all);

 private:
  template <typename T> void prepare_t();
  template <typename T> void fill_tables_t();
  template <typename T> void launch_filter_t();
  void set_units(const std::vector<kss_solver_s*>& us);
  void run_filter();
  void decide(kss_solver_s* s);
  void drop_graph();

  std::vector<kss_solver_s*> units;
  std::vector<Roles> roles;
  bool prepared = false;
  std::vector<RegPlanHost> plans;
  std::vector<PassClass> classes;
  std::vector<int> pos;  // position of each unit in the class-ordered item table
  std::vector<const void*> vpi;  // per unit: V in the CTA-wide pass B's layout (null: per-warp form)
  std::vector<WsOff> ws_off;
  DevBuf ws, d_local, d_cn, d_nn;
  std::vector<unsigned char> h_local;
  std::vector<GemmItem> h_cn, h_nn;
  size_t litem_bytes = 0;
  int scr_warp = 0;
  size_t smem_ac = 0, smem_b = 0;
  int blocks_ac = 0, blocks_b = 0;
  int cn_blocks = 0, cn_rblocks = 0, nn_blocks = 0;
  int steps = 0;
  int cur_degree = 10;
  std::vector<int> udeg;  // effective filter degree of every unit this iteration
  void* gexec = nullptr;  // cudaGraphExec_t of the captured filter
  // Worker contexts (own stream, cuSOLVER handle and GEMM workspace) that run the units'
  // Rayleigh-Ritz steps concurrently.
  std::vector<kss_ctx> workers;
  std::vector<void*> wev;  // cudaEvent_t per worker (join)
  void* fork_ev = nullptr;
  void rr_all(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
              const std::vector<int>& hy, const std::vector<int>& xo, const std::vector<int>& hxo);
  // Batched FP64 Rayleigh-Ritz of all units: matrices padded to one size, batched Cholesky,
  // triangular solves and Hermitian eigensolve (one call each for every unit).
  void rr_batched(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
                  const std::vector<int>& hy, const std::vector<int>& xo, const std::vector<int>& hxo);
  // Single precision: the projector products of every unit as grouped split-BF16 products on the
  // tensor cores (one persistent launch each for beta^H psi and beta C'); unit u is product tc_i[u]
  // of both plans (-1: no projectors).
  bool tc_on = false;
  bool simt_on = true;  // the FP32 CUDA-core grouped products run (no tensor-core plan, or units with
                        // proj32 set)
  TcGroupPlan tc_cn, tc_nn;
  std::vector<int> tc_i;
  void rr_batched_grouped(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
                          const std::vector<int>& hy, const std::vector<int>& xo, const std::vector<int>& hxo,
                          int np);
  DevBuf Sb, Hb, Wb, binfo, q32;
  // Grouped Rayleigh-Ritz of single-precision units: device tables (Gram and rotation products,
  // per-unit conversion / residual items), split-K partial sums, and a pinned staging buffer for
  // the tables (rewritten only after the stream synchronisation that ends every iteration).
  DevBuf d_rr_g, d_rr_rot, d_rr_it, rr_part;
  void* hstage = nullptr;
  size_t hstage_bytes = 0;
  void* stage(size_t bytes);
  std::vector<int> binfo_h;
  void* cap = nullptr;    // cudaStream_t used only to record the graph
};

}  // namespace kss
