// Hybrid FNO-LBM driver (Sec. 2.3, Fig. 3 of arXiv 2604.27158) and its C ABI.
//
//  steady   (Fig. 3a): FNO prediction of (rho - 1, u) from the mask and the
//           default fields -> clamp -> re-initialisation of f -> LBM time
//           marching until every grid's residual is below tol.
//  unsteady (Fig. 3b): super-time-stepping cycles of k LBM steps, m FNO steps
//           on the macroscopic fields and re-initialisation of f.  One cycle is
//           captured as a CUDA graph (one per starting buffer parity) and
//           replayed, so a cycle costs one graph launch on the host.
// Grids of equal size form one FNO batch.  All buffers live in the caller's
// workspace; the only host synchronisation is the steady residual check.
#include <math.h>

#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"
#include "lbm_internal.cuh"

namespace lbmfno {

// A size group: the grids of one (ny, nx), predicted by one FNO call per network.  Each
// group has its own FNO buffers and streams, so that the groups of an FNO step (and the
// two networks of a group) run as parallel branches.
struct Group {
  int H, W;                 // ny, nx of its grids
  std::vector<int> grids;   // grid indices
  int* grids_d = nullptr;   // device copy (workspace)
  // workspace offsets: inputs of the density (or single) and velocity networks, outputs,
  // FNO workspaces (bytes)
  size_t fin = 0, fin_u = 0, fout = 0, fout_u = 0, fws = 0, fws_u = 0;
  size_t fws_bytes = 0, fws_u_bytes = 0;
  cudaStream_t st = nullptr, st_u = nullptr;  // the group's chain; its velocity network
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
};

struct HybWs {
  size_t rho, ux, uy, tables, total;
};

// Input planes selected by a channel mask (bit 0 rho - 1, 1 u_x, 2 u_y, 3 mask; 0 = all).
static int channel_mask(int m) { return m == 0 ? 0xF : m; }
static int channel_count(int m) {
  m = channel_mask(m);
  return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1);
}

static void make_groups(const lbm_grid* grids, int ngrids, std::vector<Group>* groups) {
  std::map<std::pair<int, int>, int> at;
  groups->clear();
  for (int g = 0; g < ngrids; ++g) {
    const auto key = std::make_pair(grids[g].ny, grids[g].nx);
    auto it = at.find(key);
    if (it == at.end()) {
      at[key] = (int)groups->size();
      Group gr;
      gr.H = grids[g].ny;
      gr.W = grids[g].nx;
      groups->push_back(gr);
      it = at.find(key);
    }
    (*groups)[it->second].grids.push_back(g);
  }
}

static int plan_ws(const lbm_grid* grids, int ngrids, const fno_config* cfg,
                   const fno_config* cfg_u, HybWs* w, std::vector<Group>* groups) {
  LBM_REQUIRE(grids && ngrids > 0 && cfg, "hybrid: bad arguments");
  make_groups(grids, ngrids, groups);
  size_t cells = 0;
  for (int g = 0; g < ngrids; ++g) cells += (size_t)grids[g].nx * grids[g].ny;
  LBM_REQUIRE(cfg->c_in <= 4 && cfg->c_out <= 3 && (!cfg_u || (cfg_u->c_in <= 4 && cfg_u->c_out <= 3)),
              "hybrid: the networks read at most the 4 planes (rho-1, ux, uy, mask) and "
              "write at most (rho-1, ux, uy)");
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t a = p;
    p = align_up(p + bytes, 256);
    return a;
  };
  w->rho = take(cells * sizeof(float));
  w->ux = take(cells * sizeof(float));
  w->uy = take(cells * sizeof(float));
  for (Group& gr : *groups) {  // every group's own buffers: the groups run side by side
    const size_t gc = gr.grids.size() * (size_t)gr.H * gr.W;
    fno_sizes fs;
    LBM_TRY(fno_query(cfg, (int)gr.grids.size(), gr.H, gr.W, &fs));
    gr.fws_bytes = fs.ws_bytes;
    gr.fin = take(gc * 4 * sizeof(float));
    gr.fout = take(gc * 3 * sizeof(float));
    gr.fws = take(gr.fws_bytes);
    if (cfg_u) {
      LBM_TRY(fno_query(cfg_u, (int)gr.grids.size(), gr.H, gr.W, &fs));
      gr.fws_u_bytes = fs.ws_bytes;
      gr.fin_u = take(gc * 4 * sizeof(float));
      gr.fout_u = take(gc * 2 * sizeof(float));
      gr.fws_u = take(gr.fws_u_bytes);
    }
  }
  w->tables = take((size_t)ngrids * (sizeof(int) + sizeof(long long)) + 256);
  w->total = p;
  return LBM_OK;
}

// FNO input of a size group: the planes of (rho - 1, u_x, u_y, mask) selected by
// `chans` (bit mask, see channel_mask), in that order, per grid.
__global__ void k_pack(const GridDev* __restrict__ gd, const int* __restrict__ gids, int B, int H,
                       int W, const uint32_t* __restrict__ mask, const float* __restrict__ rho,
                       const float* __restrict__ ux, const float* __restrict__ uy, int chans,
                       float* __restrict__ in) {
  const size_t n = (size_t)B * H * W;
  const int nch = (chans & 1) + ((chans >> 1) & 1) + ((chans >> 2) & 1) + ((chans >> 3) & 1);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((size_t)H * W));
    const int c = (int)(t % ((size_t)H * W));
    const int y = c / W, x = c % W;
    const GridDev& G = gd[gids[b]];
    const long long k = G.cell_off + c;
    const size_t plane = (size_t)H * W;
    float* o = in + (size_t)b * nch * plane + c;
    int q = 0;
    if (chans & 1) o[(q++) * plane] = rho[k] - 1.0f;
    if (chans & 2) o[(q++) * plane] = ux[k];
    if (chans & 4) o[(q++) * plane] = uy[k];
    if (chans & 8) o[(q++) * plane] = (float)mask_bit(mask + G.mask_off, G.wpr, x, y);
  }
}

// FNO output -> clamped dense fields.  fields: 0 = (rho - 1, u_x, u_y) from 3 planes,
// 1 = rho - 1 from 1 plane (density network), 2 = (u_x, u_y) from 2 planes (velocity
// network).  rho = clamp(1 + out), |u| <= u_clamp.
__global__ void k_unpack(const GridDev* __restrict__ gd, const int* __restrict__ gids, int B,
                         int H, int W, const float* __restrict__ out, int fields, float rho_lo,
                         float rho_hi, float u_clamp, float* __restrict__ rho,
                         float* __restrict__ ux, float* __restrict__ uy) {
  const size_t n = (size_t)B * H * W;
  const int nch = fields == 0 ? 3 : (fields == 1 ? 1 : 2);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((size_t)H * W));
    const int c = (int)(t % ((size_t)H * W));
    const GridDev& G = gd[gids[b]];
    const long long k = G.cell_off + c;
    const size_t plane = (size_t)H * W;
    const float* o = out + (size_t)b * nch * plane + c;
    if (fields != 2) rho[k] = fminf(fmaxf(1.0f + o[0], rho_lo), rho_hi);
    if (fields != 1) {
      const int q = fields == 0 ? 1 : 0;
      float vx = o[q * plane], vy = o[(q + 1) * plane];
      const float sp = sqrtf(vx * vx + vy * vy);
      if (sp > u_clamp) {
        const float sc = u_clamp / sp;
        vx *= sc;
        vy *= sc;
      }
      ux[k] = vx;
      uy[k] = vy;
    }
  }
}

__global__ void k_fill_rest(float* __restrict__ rho, float* __restrict__ ux, float* __restrict__ uy,
                            size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    rho[t] = 1.0f;
    ux[t] = 0.0f;
    uy[t] = 0.0f;
  }
}

}  // namespace lbmfno

using namespace lbmfno;

struct hybrid_handle {
  lbm_handle* lbm = nullptr;
  fno_handle* fno = nullptr;    // single network, or the density network
  fno_handle* fno_u = nullptr;  // velocity network (may be null)
  hybrid_config cfg{};
  fno_config fcfg{}, fcfg_u{};
  std::vector<Group> groups;
  HybWs w{};
  char* ws = nullptr;
  float *rho = nullptr, *ux = nullptr, *uy = nullptr;
  cudaStream_t cap = nullptr;     // private stream used for graph capture and replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_fno = nullptr;   // start of an FNO step (the groups' branches wait on it)
  cudaGraphExec_t cycle[2] = {nullptr, nullptr};  // by starting buffer parity
};

static inline cudaStream_t HS(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// FNO prediction for every size group from the dense fields, clamped into the same fields.
// A group's chain (pack, FNO, write-back) reads and writes only its own grids' cells, so
// the groups run as parallel branches (their own streams, forked from and joined back into
// `s` by events, which a stream capture turns into graph edges).  With two networks both
// inputs of a group are packed before either output is written back, so both read the
// fields of the same time level; the velocity network runs on a further branch while the
// density network and its write-back (rho only) run on the group's chain, which waits for
// it before writing u back.
static int hyb_predict(hybrid_handle* h, cudaStream_t s) {
  lbm_handle* L = h->lbm;
  const float lo = (float)h->cfg.rho_lo, hi = (float)h->cfg.rho_hi, uc = (float)h->cfg.u_clamp;
  LBM_CHECK_CUDA(cudaEventRecord(h->ev_fno, s));
  for (Group& gr : h->groups) {
    const int B = (int)gr.grids.size();
    const size_t n = (size_t)B * gr.H * gr.W;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 65535);
    float* fin = reinterpret_cast<float*>(h->ws + gr.fin);
    float* fout = reinterpret_cast<float*>(h->ws + gr.fout);
    float* fin_u = reinterpret_cast<float*>(h->ws + gr.fin_u);
    float* fout_u = reinterpret_cast<float*>(h->ws + gr.fout_u);
    cudaStream_t cs = gr.st;
    LBM_CHECK_CUDA(cudaStreamWaitEvent(cs, h->ev_fno, 0));
    k_pack<<<blocks, 256, 0, cs>>>(L->gd_d, gr.grids_d, B, gr.H, gr.W, L->mask, h->rho, h->ux,
                                   h->uy, channel_mask(h->cfg.in_channels), fin);
    LBM_CHECK_LAUNCH();
    if (h->fno_u) {
      k_pack<<<blocks, 256, 0, cs>>>(L->gd_d, gr.grids_d, B, gr.H, gr.W, L->mask, h->rho, h->ux,
                                     h->uy, channel_mask(h->cfg.in_channels_u), fin_u);
      LBM_CHECK_LAUNCH();
      LBM_CHECK_CUDA(cudaEventRecord(gr.ev_fork, cs));  // fork: the velocity network
      LBM_CHECK_CUDA(cudaStreamWaitEvent(gr.st_u, gr.ev_fork, 0));
      LBM_TRY(fno_forward(h->fno_u, fin_u, fout_u, B, gr.H, gr.W, h->ws + gr.fws_u,
                          gr.fws_u_bytes, gr.st_u));
      LBM_CHECK_CUDA(cudaEventRecord(gr.ev_join, gr.st_u));
    }
    LBM_TRY(fno_forward(h->fno, fin, fout, B, gr.H, gr.W, h->ws + gr.fws, gr.fws_bytes, cs));
    k_unpack<<<blocks, 256, 0, cs>>>(L->gd_d, gr.grids_d, B, gr.H, gr.W, fout,
                                     h->fno_u ? 1 : 0, lo, hi, uc, h->rho, h->ux, h->uy);
    LBM_CHECK_LAUNCH();
    if (h->fno_u) {  // join
      LBM_CHECK_CUDA(cudaStreamWaitEvent(cs, gr.ev_join, 0));
      k_unpack<<<blocks, 256, 0, cs>>>(L->gd_d, gr.grids_d, B, gr.H, gr.W, fout_u, 2, lo, hi, uc,
                                       h->rho, h->ux, h->uy);
      LBM_CHECK_LAUNCH();
    }
    LBM_CHECK_CUDA(cudaEventRecord(gr.ev_done, cs));
    LBM_CHECK_CUDA(cudaStreamWaitEvent(s, gr.ev_done, 0));
  }
  return LBM_OK;
}

// One unsteady cycle: k LBM steps, m FNO steps, re-initialisation.
static int hyb_cycle(hybrid_handle* h, cudaStream_t s) {
  LBM_TRY(lbm_step(h->lbm, h->cfg.k_lbm, s));
  LBM_TRY(lbm_macro(h->lbm, h->rho, h->ux, h->uy, s));
  for (int j = 0; j < h->cfg.m_fno; ++j) LBM_TRY(hyb_predict(h, s));
  return lbm_reinit_from_macro(h->lbm, h->rho, h->ux, h->uy, h->cfg.neq_mode, s);
}

extern "C" {

int hybrid_query_ws(const lbm_grid* grids_h, int ngrids, const fno_config* cfg_h,
                    const fno_config* cfg_u_h, size_t* ws_h) {
  LBM_REQUIRE(ws_h != nullptr, "hybrid_query_ws: null output");
  HybWs w;
  std::vector<Group> groups;
  LBM_TRY(plan_ws(grids_h, ngrids, cfg_h, cfg_u_h, &w, &groups));
  *ws_h = w.total;
  return LBM_OK;
}

int hybrid_create(lbm_handle* lbm, fno_handle* fno, fno_handle* fno_u, const hybrid_config* cfg_h,
                  void* ws_d, size_t ws_bytes, hybrid_handle** out) {
  LBM_REQUIRE(out != nullptr, "hybrid_create: null handle output");
  *out = nullptr;
  LBM_REQUIRE(lbm && cfg_h && ws_d, "hybrid_create: null argument");
  LBM_REQUIRE(((uintptr_t)ws_d % 256) == 0, "hybrid_create: workspace must be 256-byte aligned");
  const hybrid_config& c = *cfg_h;
  LBM_REQUIRE(c.mode == HYBRID_STEADY || c.mode == HYBRID_UNSTEADY, "hybrid_create: bad mode");
  if (c.mode == HYBRID_STEADY)
    LBM_REQUIRE(c.check_every >= 1 && c.tol > 0 && c.max_steps >= 1,
                "hybrid_create: steady mode needs check_every >= 1, tol > 0, max_steps >= 1");
  else
    LBM_REQUIRE(c.k_lbm >= 0 && c.m_fno >= 0 && fno, "hybrid_create: unsteady mode needs an FNO");
  const bool needs_fno = (c.mode == HYBRID_UNSTEADY && c.m_fno > 0) ||
                         (c.mode == HYBRID_STEADY && c.use_fno);
  LBM_REQUIRE(!needs_fno || fno, "hybrid_create: this configuration needs an FNO handle");
  LBM_REQUIRE(c.rho_lo > 0.0 && c.rho_hi > c.rho_lo && c.u_clamp > 0.0,
              "hybrid_create: bad clamp bounds");
  LBM_REQUIRE(c.in_channels >= 0 && c.in_channels <= 0xF && c.in_channels_u >= 0 &&
                  c.in_channels_u <= 0xF,
              "hybrid_create: in_channels must be a 4-bit plane mask");
  LBM_REQUIRE(!fno_u || fno, "hybrid_create: a velocity network needs a density network");
  fno_config fc{}, fcu{};
  if (fno) {
    LBM_TRY(fno_get_config(fno, &fc));
    LBM_REQUIRE(fc.c_in == channel_count(c.in_channels),
                "hybrid_create: the network reads %d planes, in_channels selects %d", fc.c_in,
                channel_count(c.in_channels));
    LBM_REQUIRE(fc.c_out == (fno_u ? 1 : 3),
                "hybrid_create: the %s network must have %d output channels",
                fno_u ? "density" : "single", fno_u ? 1 : 3);
  } else {
    fc = fno_config{4, 3, 2, 1, 1, 1, 1, FNO_ACT_GELU, 0};
  }
  if (fno_u) {
    LBM_TRY(fno_get_config(fno_u, &fcu));
    LBM_REQUIRE(fcu.c_in == channel_count(c.in_channels_u),
                "hybrid_create: the velocity network reads %d planes, in_channels_u selects %d",
                fcu.c_in, channel_count(c.in_channels_u));
    LBM_REQUIRE(fcu.c_out == 2, "hybrid_create: the velocity network must have 2 outputs");
  }
  hybrid_handle* h = new hybrid_handle();
  h->lbm = lbm;
  h->fno = fno;
  h->fno_u = fno_u;
  h->cfg = c;
  h->fcfg = fc;
  h->fcfg_u = fcu;
  int st = plan_ws(lbm->grids.data(), lbm->ngrids, &fc, fno_u ? &fcu : nullptr, &h->w,
                   &h->groups);
  if (st == LBM_OK && ws_bytes < h->w.total) {
    set_error("hybrid_create: workspace too small (%zu < %zu)", ws_bytes, h->w.total);
    st = LBM_ERR_INVALID_ARG;
  }
  if (st != LBM_OK) {
    delete h;
    return st;
  }
  h->ws = static_cast<char*>(ws_d);
  h->rho = reinterpret_cast<float*>(h->ws + h->w.rho);
  h->ux = reinterpret_cast<float*>(h->ws + h->w.ux);
  h->uy = reinterpret_cast<float*>(h->ws + h->w.uy);
  // per-group index / offset tables
  std::vector<int> ids;
  int* ids_d = reinterpret_cast<int*>(h->ws + h->w.tables);
  for (Group& gr : h->groups) {
    gr.grids_d = ids_d + ids.size();
    for (int g : gr.grids) ids.push_back(g);
  }
  if (cudaMemcpy(ids_d, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fno, cudaEventDisableTiming) != cudaSuccess ||
      !std::all_of(h->groups.begin(), h->groups.end(), [](Group& gr) {
        return cudaStreamCreateWithFlags(&gr.st, cudaStreamNonBlocking) == cudaSuccess &&
               cudaStreamCreateWithFlags(&gr.st_u, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&gr.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&gr.ev_join, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&gr.ev_done, cudaEventDisableTiming) == cudaSuccess;
      })) {
    set_error("hybrid_create: %s", cudaGetErrorString(cudaGetLastError()));
    hybrid_destroy(h);
    return LBM_ERR_CUDA;
  }
  *out = h;
  return LBM_OK;
}

int hybrid_advance(hybrid_handle* h, int cycles, hybrid_stats* out_h, int64_t* grid_steps_h,
                   double* grid_residual_h, void* stream) {
  LBM_REQUIRE(h != nullptr, "hybrid_advance: null handle");
  cudaStream_t s = HS(stream);
  lbm_handle* L = h->lbm;
  hybrid_stats stats{};
  const hybrid_config& c = h->cfg;
  if (c.mode == HYBRID_STEADY) {
    const size_t cells = L->layout.cells;
    const unsigned blocks = (unsigned)std::min<size_t>((cells + 255) / 256, 65535);
    k_fill_rest<<<blocks, 256, 0, s>>>(h->rho, h->ux, h->uy, cells);
    LBM_CHECK_LAUNCH();
    if (c.use_fno) {
      LBM_TRY(hyb_predict(h, s));
      stats.fno_calls = (int)h->groups.size() * (h->fno_u ? 2 : 1);
    }
    LBM_TRY(lbm_reinit_from_macro(L, h->rho, h->ux, h->uy, c.use_fno ? c.neq_mode : 0, s));
    const int ng = L->ngrids;
    std::vector<int64_t> first(ng, -1);
    std::vector<double> st((size_t)ng * LBM_NSTAT);
    long long steps = 0;
    bool all = false;
    // A check takes the statistics of level `steps` inside the step kernel that writes
    // level steps + 1 into the other buffer; that step is kept (it is the first step of
    // the next interval) unless the loop ends at this check.
    int carried = 0;
    while (steps < c.max_steps) {
      const int k = (int)std::min<long long>(c.check_every, c.max_steps - steps);
      LBM_TRY(lbm_step(L, k - carried, s));
      steps += k;
      LBM_TRY(residual_step(L, st.data(), 1, s));
      carried = 0;
      all = true;
      double mx = 0.0;
      for (int g = 0; g < ng; ++g) {
        const double r = st[(size_t)g * LBM_NSTAT + LBM_STAT_RESIDUAL];
        if (first[g] < 0 && r < c.tol) first[g] = steps;
        if (first[g] < 0) all = false;
        mx = std::max(mx, r);
      }
      stats.max_residual = mx;
      if (all || steps >= c.max_steps) break;
      accept_step(L);
      carried = 1;
    }
    stats.steps = steps;
    stats.converged = all ? 1 : 0;
    for (int g = 0; g < ng; ++g) {
      if (grid_steps_h) grid_steps_h[g] = first[g];
      if (grid_residual_h) grid_residual_h[g] = st[(size_t)g * LBM_NSTAT + LBM_STAT_RESIDUAL];
    }
  } else {
    LBM_REQUIRE(cycles >= 0, "hybrid_advance: cycles must be >= 0");
    // order the private stream after the caller's work
    LBM_CHECK_CUDA(cudaEventRecord(h->ev_in, s));
    LBM_CHECK_CUDA(cudaStreamWaitEvent(h->cap, h->ev_in, 0));
    for (int k = 0; k < cycles; ++k) {
      const int parity = L->cur;
      if (!h->cycle[parity]) {
        cudaGraph_t g = nullptr;
        LBM_CHECK_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        const long long steps_before = L->steps;
        const int rc = hyb_cycle(h, h->cap);
        const cudaError_t ec = cudaStreamEndCapture(h->cap, &g);
        if (rc != LBM_OK) return rc;
        LBM_CHECK_CUDA(ec);
        LBM_CHECK_CUDA(cudaGraphInstantiate(&h->cycle[parity], g, 0));
        cudaGraphDestroy(g);
        L->cur = parity;  // capture recorded the launches without running them
        L->steps = steps_before;
      }
      LBM_CHECK_CUDA(cudaGraphLaunch(h->cycle[parity], h->cap));
      if (c.k_lbm % 2) L->cur ^= 1;
      L->steps = 0;  // the cycle ends with a re-initialisation
      stats.steps += c.k_lbm;
      stats.fno_calls += c.m_fno * (int)h->groups.size() * (h->fno_u ? 2 : 1);
    }
    LBM_CHECK_CUDA(cudaEventRecord(h->ev_out, h->cap));
    LBM_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_out, 0));
  }
  if (out_h) *out_h = stats;
  return LBM_OK;
}

int hybrid_destroy(hybrid_handle* h) {
  if (!h) return LBM_OK;
  for (int p = 0; p < 2; ++p)
    if (h->cycle[p]) cudaGraphExecDestroy(h->cycle[p]);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_fno) cudaEventDestroy(h->ev_fno);
  for (Group& gr : h->groups) {
    for (cudaEvent_t e : {gr.ev_fork, gr.ev_join, gr.ev_done})
      if (e) cudaEventDestroy(e);
    if (gr.st) cudaStreamDestroy(gr.st);
    if (gr.st_u) cudaStreamDestroy(gr.st_u);
  }
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
  return LBM_OK;
}

}  // extern "C"
