// C ABI of libgnntrk: handle life cycle, weight upload, workspace and the
// launch sequence of the hot path. See include/gnntrk.h for the contract.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gnntrk.h"
#include "internal.cuh"
#include "tc.cuh"

using namespace gnntrk;

namespace gnntrk {
int device_sms();
}

struct gnntrk_handle {
  gnntrk_cfg cfg{};
  int device = 0;
  int D = 0, h = 0, K = 0, n_embed = 0;
  // FP32 weights (SIMT layout)
  float* d_wf32 = nullptr;
  LayerF32 embed[kMaxEmbedLayers]{};
  Mlp2F32 node_enc{}, edge_enc{}, cls{}, node[kMaxIters]{}, edge[kMaxIters]{};
  // INT8 embedding: packed weights, scales, the ranges set by the caller
  Int8Embed i8{};
  void* d_i8 = nullptr;
  std::vector<std::vector<float>> i8_sw;  // per layer: weight scales S_w
  std::vector<float> i8_alpha;            // per layer: input range
  EmbedAmax amax_layers{};
  int32_t* d_amax = nullptr;
  TripletHeads trip{};   // triplet classifiers (blob with triplet layers)
  bool has_trip = false;
  TrackOut track_out{};  // outputs of the current triplet call
  bool want_tracks = false;
  EdgeProj enc_proj{}, step_proj[kMaxIters]{};  // h_src / h_dst column blocks
  // tensor-core weights (BF16 / FP8 packed operands)
  TcModel tc{};
  void* d_wtc = nullptr;
  void* d_wtrip = nullptr;  // triplet-classifier images (tensor-core paths)
  // workspace
  Ws ws{};
  std::vector<void*> allocs;
  // last call
  int last_events = 0, last_hits = 0;
  int last_launches = 0;
  cudaStream_t last_stream = nullptr;
  std::string err;
  // per-stage profiling
  bool profiling = false;
  struct StageAcc {
    std::string name;
    double ms = 0.0;
    int64_t runs = 0;
  };
  std::vector<StageAcc> stages;
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  // CUDA graphs of earlier call shapes (use_graph)
  struct GraphEntry {
    int32_t n_events;
    int64_t n_hits;
    const void *xyz, *plane, *offsets, *labels;
    const void *ev_tracks, *track_off, *track_hits;
    int64_t max_tracks, max_track_hits;
    cudaGraphExec_t exec;
    int launches;
  };
  std::vector<GraphEntry> graphs;
};

namespace {

thread_local std::string g_create_error;  // per host thread, like errno

gnntrk_status fail(gnntrk_handle* h, gnntrk_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

gnntrk_status cuda_fail(gnntrk_handle* h, cudaError_t e, const char* what) {
  return fail(h, GNNTRK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

uint32_t rd_u32(const unsigned char* p) {
  return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) | (uint32_t(p[3]) << 24);
}

// Parse and shape-check the weight blob.
bool parse_weights(const void* blob, size_t n, const gnntrk_cfg& c, std::vector<HostLayer>& L,
                   std::string& why) {
  const unsigned char* p = static_cast<const unsigned char*>(blob);
  if (!blob || n < 16) return why = "weight blob too short", false;
  if (rd_u32(p) != 0x57544E47u) return why = "weight blob: bad magic", false;
  if (rd_u32(p + 4) != 1u) return why = "weight blob: unsupported version", false;
  const uint32_t nl = rd_u32(p + 8);
  std::vector<std::pair<int, int>> want;
  for (int l = 0; l < c.n_embed_layers; ++l) want.push_back({c.embed_dims[l], c.embed_dims[l + 1]});
  const int h = c.hidden;
  want.push_back({3, h});
  want.push_back({h, h});
  want.push_back({2 * h, h});
  want.push_back({h, h});
  for (int k = 0; k < c.iters; ++k) {
    want.push_back({3 * h, h});
    want.push_back({h, h});
    want.push_back({3 * h, h});
    want.push_back({h, h});
  }
  want.push_back({h, h});
  want.push_back({h, 1});
  // optional triplet classifiers (articulation, elbow): 2h -> h -> 1 each
  if (nl == want.size() + 4)
    for (int t = 0; t < 2; ++t) {
      want.push_back({2 * h, h});
      want.push_back({h, 1});
    }
  if (nl != want.size()) return why = "weight blob: layer count does not match cfg", false;
  if (n < 16 + 8 * size_t(nl)) return why = "weight blob: truncated header", false;
  size_t need = 16 + 8 * size_t(nl);
  L.resize(nl);
  for (uint32_t l = 0; l < nl; ++l) {
    L[l].in = int(rd_u32(p + 16 + 8 * l));
    L[l].out = int(rd_u32(p + 20 + 8 * l));
    if (L[l].in != want[l].first || L[l].out != want[l].second)
      return why = "weight blob: layer " + std::to_string(l) + " shape does not match cfg", false;
    need += 4 * (size_t(L[l].in) * L[l].out + L[l].out);
  }
  if (n != need) return why = "weight blob: size does not match its header", false;
  size_t off = 16 + 8 * size_t(nl);
  for (uint32_t l = 0; l < nl; ++l) {
    L[l].W.resize(size_t(L[l].in) * L[l].out);
    L[l].b.resize(L[l].out);
    std::memcpy(L[l].W.data(), p + off, 4 * L[l].W.size());
    off += 4 * L[l].W.size();
    std::memcpy(L[l].b.data(), p + off, 4 * L[l].b.size());
    off += 4 * L[l].b.size();
  }
  return true;
}

gnntrk_status alloc(gnntrk_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, GNNTRK_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  h->allocs.push_back(*p);
  return GNNTRK_OK;
}

template <class T>
gnntrk_status alloc_n(gnntrk_handle* h, T** p, size_t n) {
  return alloc(h, reinterpret_cast<void**>(p), n * sizeof(T));
}

gnntrk_status upload_f32(gnntrk_handle* h, const std::vector<HostLayer>& L) {
  std::vector<float> img;
  std::vector<size_t> wofs(L.size()), bofs(L.size());
  std::vector<int> ldo(L.size());
  for (size_t l = 0; l < L.size(); ++l) {
    ldo[l] = (L[l].out + 3) & ~3;
    wofs[l] = img.size();
    img.resize(img.size() + size_t(L[l].in) * ldo[l], 0.f);
    for (int o = 0; o < L[l].out; ++o)
      for (int i = 0; i < L[l].in; ++i)
        img[wofs[l] + size_t(i) * ldo[l] + o] = L[l].W[size_t(o) * L[l].in + i];
    bofs[l] = img.size();
    img.resize(img.size() + ldo[l], 0.f);
    for (int o = 0; o < L[l].out; ++o) img[bofs[l] + o] = L[l].b[o];
  }
  // a zero bias for the projection views
  const size_t zofs = img.size();
  img.resize(img.size() + size_t((h->h + 3) & ~3) + 4, 0.f);
  gnntrk_status st = alloc_n(h, &h->d_wf32, img.size());
  if (st) return st;
  cudaError_t e = cudaMemcpy(h->d_wf32, img.data(), img.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "weight upload");
  auto lay = [&](size_t l) {
    return LayerF32{h->d_wf32 + wofs[l], h->d_wf32 + bofs[l], L[l].in, L[l].out, ldo[l]};
  };
  size_t c = 0;
  for (int l = 0; l < h->n_embed; ++l) h->embed[l] = lay(c++);
  h->node_enc = {lay(c), lay(c + 1)};
  c += 2;
  h->edge_enc = {lay(c), lay(c + 1)};
  c += 2;
  for (int k = 0; k < h->K; ++k) {
    h->node[k] = {lay(c), lay(c + 1)};
    h->edge[k] = {lay(c + 2), lay(c + 3)};
    c += 4;
  }
  h->cls = {lay(c), lay(c + 1)};
  if (L.size() == c + 6) {
    h->trip.art = {lay(c + 2), lay(c + 3)};
    h->trip.elb = {lay(c + 4), lay(c + 5)};
    h->has_trip = true;
  }
  // projection views: rows [k0, k0 + h) of a transposed first layer
  const float* zero = h->d_wf32 + zofs;
  auto view = [&](const LayerF32& l1, int k0) {
    return LayerF32{l1.WT + size_t(k0) * l1.ldo, zero, h->h, l1.out, l1.ldo};
  };
  h->enc_proj = {view(h->edge_enc.l1, 0), view(h->edge_enc.l1, h->h)};
  for (int k = 0; k < h->K; ++k) h->step_proj[k] = {view(h->edge[k].l1, h->h), view(h->edge[k].l1, 2 * h->h)};
  return GNNTRK_OK;
}

// Every workspace array with its size in bytes (one list for allocation and
// for gnntrk_workspace_bytes).
std::vector<std::pair<void**, size_t>> workspace_plan(const gnntrk_cfg& c, int D, int hd, Ws& w) {
  const int64_t H = c.max_hits, E = int64_t(c.max_hits) * c.edges_per_hit;
  std::vector<std::pair<void**, size_t>> v;
  auto add = [&](auto** ptr, int64_t n) {
    v.push_back({reinterpret_cast<void**>(ptr), size_t(n) * sizeof(**ptr)});
  };
  add(&w.perm, H);
  add(&w.node_event, H);
  add(&w.pos, H);
  add(&w.plane_off, int64_t(c.max_events) * (c.n_planes + 1));
  add(&w.emb, H * D);
  add(&w.deg, H);
  add(&w.graph_desc, c.max_events);
  add(&w.row_ptr, H + 1);
  add(&w.col, E);
  add(&w.src, E);
  add(&w.d2, E);
  add(&w.in_cnt, H);
  add(&w.in_ptr, H + 1);
  add(&w.in_edge, E);
  add(&w.hstate, H * hd);
  add(&w.estate, E * hd);
  add(&w.pstate, H * 2 * hd);
  if (c.precision == GNNTRK_FP8_E4M3 && hd == 128) add(&w.hamax, H);
  if (c.precision != GNNTRK_FP32) {
    add(&w.hstate16, H * hd);
    add(&w.estate16, E * hd);
  }
  add(&w.logit, E);
  add(&w.keep, E);
  add(&w.parent, H);
  add(&w.counters, C_COUNT);
  add(&w.scan_blocks, (H + 4095) / 4096 + 1);
  add(&w.ev_off, int64_t(c.max_events) + 1);
  if (c.precision != GNNTRK_FP32) {
    add(&w.rs_elev, E);
    add(&w.rs_nlev, H);
    add(&w.rs_elist, E * (c.iters + 1));
    add(&w.rs_nlist, H * (c.iters + 1));
    add(&w.rs_counts, 6 * (kMaxIters + 2));
    add(&w.rs_desc, int64_t(c.max_events) * (1 + 4 * (kMaxIters + 1)));
  }
  const int64_t T = c.triplets ? H * c.triplets_per_hit : 0;
  if (c.triplets) {
    add(&w.trip_cnt_a, H);
    add(&w.trip_cnt_e, H);
    add(&w.trip_off_a, H + 1);
    add(&w.trip_off_e, H + 1);
    add(&w.trip_a1, T);
    add(&w.trip_a2, T);
    add(&w.trip_alogit, T);
    add(&w.trip_akeep, T);
    add(&w.trip_e1, T);
    add(&w.trip_e2, T);
    add(&w.trip_et, T);
    add(&w.trip_elogit, T);
    add(&w.trip_ekeep, T);
    add(&w.tb_par, E);
    add(&w.tb_par2, E);
    add(&w.tb_out, E);
    add(&w.tb_in, E);
    add(&w.tb_flag, E);
    add(&w.tb_cnt, E);
    add(&w.tb_off, E);
    add(&w.tb_cur, E);
    add(&w.tb_hits, 2 * E);
    add(&w.tb_pairs, T);
    add(&w.tb_ev_tracks, c.max_events);
    add(&w.tb_ev_hits, c.max_events);
    add(&w.tb_ev_pairs, c.max_events);
    add(&w.tb_ev_hit_off, int64_t(c.max_events) + 1);
  }
  w.h_cap = H;
  w.e_cap = E;
  w.t_cap = T;
  return v;
}

gnntrk_status alloc_workspace(gnntrk_handle* h) {
  auto plan = workspace_plan(h->cfg, h->D, h->h, h->ws);
  for (auto& it : plan) {
    gnntrk_status st = alloc(h, it.first, it.second);
    if (st) return st;
  }
  cudaMemset(h->ws.counters, 0, C_COUNT * sizeof(int32_t));
  return GNNTRK_OK;
}

GraphParams graph_params(const gnntrk_handle* h) {
  GraphParams g{};
  g.n_planes = h->cfg.n_planes;
  g.k_max = h->cfg.k_max;
  g.radius2 = h->cfg.radius2;
  g.cut_logit = float(std::log(double(h->cfg.score_cut) / (1.0 - double(h->cfg.score_cut))));
  for (int i = 0; i < 6; ++i) g.fs[i] = h->cfg.feat_scale[i];
  return g;
}

bool valid_d(int d) { return (d >= 1 && d <= 8) || d == 16; }

cudaEvent_t take_event(gnntrk_handle* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// wait for the recorded stage events and fold them into the totals
void collect_stages(gnntrk_handle* h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->stages[p.stage].ms += ms;
      h->stages[p.stage].runs += 1;
    }
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->pending.clear();
  cudaGetLastError();
}

// Runs `fn` (which enqueues one pipeline stage on s) and, when profiling,
// brackets it with an event pair on the same stream.
template <class F>
void stage(gnntrk_handle* h, const char* name, cudaStream_t s, int kernels, F&& fn) {
  h->last_launches += kernels;
  if (!h->profiling) {
    fn();
    return;
  }
  int idx = -1;
  for (size_t i = 0; i < h->stages.size(); ++i)
    if (h->stages[i].name == name) idx = int(i);
  if (idx < 0) {
    h->stages.push_back({name, 0.0, 0});
    idx = int(h->stages.size()) - 1;
  }
  cudaEvent_t a = take_event(h), b = take_event(h);
  cudaEventRecord(a, s);
  fn();
  cudaEventRecord(b, s);
  h->pending.push_back({idx, a, b});
}

}  // namespace

// Enqueue the whole hot path of one call on stream s (also used inside a
// CUDA-graph capture).
void enqueue_pipeline(gnntrk_handle* h, const Batch& b, const int64_t* offsets, cudaStream_t s) {
  const gnntrk_cfg& c = h->cfg;
  Ws& w = h->ws;
  const GraphParams g = graph_params(h);
  if (h->profiling) collect_stages(h);
  h->last_launches = 0;
  cudaMemsetAsync(w.counters, 0, C_COUNT * sizeof(int32_t), s);
  cudaMemcpyAsync(w.ev_off, offsets, sizeof(int64_t) * (b.n_events + 1), cudaMemcpyDeviceToDevice, s);
  stage(h, "sort", s, 1, [&] { launch_sort(b, w, c.n_planes, s); });
  const Sel all{nullptr, nullptr};
  const bool tc = c.precision != GNNTRK_FP32;
  const bool i8 = c.embed_int8 != 0;
  stage(h, "node_prep", s, (tc ? 2 : 1) + (i8 ? 1 : 0) - (tc && i8 ? 1 : 0), [&] {
    if (i8) launch_embed_int8(b, w, h->i8, h->D, g, s);
    if (!tc)
      launch_node_prep_f32(b, w, h->embed, h->n_embed, h->node_enc, h->enc_proj, h->D, h->h, g,
                           !i8, true, all, s);
    else
      tc_node_prep(b, w, h->tc, h->embed, h->n_embed, h->D, h->h, g, h->node_enc.l1, s, !i8);
  });
  stage(h, "graph", s, 1, [&] { launch_graph(b, w, g, h->D, s); });
  if (!tc) {
    stage(h, "edge_encoder", s, 1, [&] { launch_edge_enc_f32(b, w, h->edge_enc, h->h, all, s); });
    for (int k = 0; k < h->K; ++k) {
      stage(h, "node_messages", s, 1, [&] { launch_messages_f32(b, w, h->h, all, s); });
      stage(h, "node_update", s, 1,
            [&] { launch_node_update_f32(b, w, h->node[k], h->step_proj[k], h->h, all, s); });
      const bool last = k + 1 == h->K;
      if (last && c.triplets) {
        // e^K stays in memory for the triplet classifiers: step, then classifier
        stage(h, "edge_update", s, 2, [&] {
          launch_edge_update_f32(b, w, h->edge[k], nullptr, h->h, g.cut_logit, false, 0.f, 0.f,
                                 all, s);
          launch_edge_update_f32(b, w, Mlp2F32{}, &h->cls, h->h, g.cut_logit, false, 0.f, 0.f,
                                 all, s);
        });
      } else {
        stage(h, "edge_update", s, 1, [&] {
          launch_edge_update_f32(b, w, h->edge[k], last ? &h->cls : nullptr, h->h, g.cut_logit,
                                 false, 0.f, 0.f, all, s);
        });
      }
    }
    if (h->K == 0)  // no message passing: the classifier reads the edge encodings
      stage(h, "edge_update", s, 1, [&] {
        launch_edge_update_f32(b, w, Mlp2F32{}, &h->cls, h->h, g.cut_logit, false, 0.f, 0.f,
                               all, s);
      });
  } else {
    const bool fused = tc_cls_fused(h->h, c.precision) && !c.triplets;
    stage(h, "edge_encoder", s, 1,
          [&] { tc_gnn(b, w, h->tc, h->h, h->K, g, h->cls.l2, s, 0); });
    for (int k = 0; k < h->K; ++k) {
      stage(h, "node_messages", s, 1,
            [&] { tc_messages(b, w, h->h, c.precision == GNNTRK_FP8_E4M3, s); });
      stage(h, "node_update", s, 1,
            [&] { tc_gnn(b, w, h->tc, h->h, h->K, g, h->cls.l2, s, 1 + 2 * k); });
      stage(h, "edge_update", s, (k + 1 == h->K && !fused) ? 2 : 1,
            [&] { tc_gnn(b, w, h->tc, h->h, h->K, g, h->cls.l2, s, 2 + 2 * k, c.triplets != 0); });
    }
    if (h->K == 0)
      stage(h, "edge_update", s, 1, [&] { tc_gnn(b, w, h->tc, h->h, h->K, g, h->cls.l2, s, 1); });
    if (c.rescore_band > 0.f) {
      const double lo = double(c.score_cut) - double(c.rescore_band);
      const double hi = double(c.score_cut) + double(c.rescore_band);
      const float band_lo = lo <= 0.0 ? -INFINITY : float(std::log(lo / (1.0 - lo)));
      const float band_hi = hi >= 1.0 ? INFINITY : float(std::log(hi / (1.0 - hi)));
      // exact receptive field of the band edges and its row lists, then FP32
      // over those rows only
      int mk = 0;
      stage(h, "rescore_field", s, 0, [&] { mk = launch_rescore_sets(b, w, band_lo, band_hi, h->K, s); });
      h->last_launches += mk;
      const int NL = kMaxIters + 2;
      const int32_t* cge_e = w.rs_counts + 2 * NL;  // [k + 1]: edges of step k
      const int32_t* cge_n = w.rs_counts + 5 * NL;  // [k + 1]: hits of step k
      // each step's rows in index order: list k + 1 of rs_elist / rs_nlist
      auto esel = [&](int k) { return Sel{w.rs_elist + size_t(k + 1) * w.e_cap, cge_e + k + 1}; };
      auto nsel = [&](int k) { return Sel{w.rs_nlist + size_t(k + 1) * w.h_cap, cge_n + k + 1}; };
      stage(h, "rescore_node_prep", s, 1, [&] {
        launch_node_prep_f32(b, w, h->embed, h->n_embed, h->node_enc, h->enc_proj, h->D, h->h, g,
                             false, true, nsel(-1), s);
      });
      stage(h, "rescore_edge_encoder", s, 1,
            [&] { launch_edge_enc_f32(b, w, h->edge_enc, h->h, esel(-1), s); });
      for (int k = 0; k < h->K; ++k) {
        stage(h, "rescore_node_messages", s, 1,
              [&] { launch_messages_f32(b, w, h->h, nsel(k), s); });
        stage(h, "rescore_node_update", s, 1, [&] {
          launch_node_update_f32(b, w, h->node[k], h->step_proj[k], h->h, nsel(k), s);
        });
        stage(h, "rescore_edge_update", s, 1, [&] {
          launch_edge_update_f32(b, w, h->edge[k], k + 1 == h->K ? &h->cls : nullptr, h->h,
                                 g.cut_logit, true, band_lo, band_hi, esel(k), s);
        });
      }
      if (h->K == 0)
        stage(h, "rescore_edge_update", s, 1, [&] {
          launch_edge_update_f32(b, w, Mlp2F32{}, &h->cls, h->h, g.cut_logit, true, band_lo,
                                 band_hi, esel(-1), s);
        });
    }
  }
  stage(h, "components", s, 1, [&] { launch_cc(b, w, s); });
  if (h->want_tracks) {
    const float tcut = float(std::log(double(c.triplet_cut) / (1.0 - double(c.triplet_cut))));
    stage(h, "triplets", s, 6, [&] { launch_triplets(b, w, h->h, s); });
    stage(h, "triplet_scores", s, 3, [&] {
      if (h->tc.has_trip) {
        // tensor cores: BF16 final edge encodings times BF16 first layers
        tc_triplet_scores(b, w, h->tc, h->h, h->trip.art.l2, h->trip.elb.l2, h->trip.art.l1.b,
                          h->trip.elb.l1.b, tcut, s);
        launch_triplet_kept(w, s);
      } else {
        launch_triplet_scores_f32(b, w, h->trip, h->h, tcut, s);
        launch_triplet_kept(w, s);
      }
    });
    stage(h, "track_build", s, 6, [&] { launch_track_build(b, w, h->track_out, s); });
  }
}

namespace {
// Upload the dequantisation scales (alpha / 127) S_w and 127 / alpha of the
// INT8 embedding for the current ranges.
gnntrk_status upload_i8_scales(gnntrk_handle* h) {
  const int n = h->n_embed;
  std::vector<float> buf;
  for (int l = 0; l < n; ++l) {
    const float sa = h->i8_alpha[l] / 127.0f;
    for (float sw : h->i8_sw[l]) buf.push_back(sa * sw);
  }
  for (int l = 0; l < n; ++l) buf.push_back(127.0f / h->i8_alpha[l]);
  float* d = const_cast<float*>(h->i8.l[0].s);
  cudaError_t e = cudaMemcpy(d, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? GNNTRK_OK : cuda_fail(h, e, "INT8 scale upload");
}

// Quantise the embedding weights per output channel and lay out the INT8
// kernel's operands: codes (4 per word along K, rows padded to whole 16-byte
// chunks), biases, then the scales.
gnntrk_status setup_int8(gnntrk_handle* h, const std::vector<HostLayer>& L) {
  const int n = h->n_embed;
  std::vector<uint32_t> words;
  std::vector<size_t> w_off(n);
  std::vector<int> in4(n), in16(n);
  h->i8_sw.assign(n, {});
  h->i8_alpha.assign(n, 1.0f);
  int max_in4 = 1;
  for (int l = 0; l < n; ++l) {
    const HostLayer& y = L[l];
    int q4 = (y.in + 3) / 4, p4 = 1;
    while (p4 < q4) p4 *= 2;
    in4[l] = p4;
    in16[l] = (p4 + 3) / 4;
    if (l > 0) max_in4 = std::max(max_in4, p4);
    w_off[l] = words.size();
    words.resize(words.size() + size_t(y.out) * in16[l] * 4, 0u);
    for (int o = 0; o < y.out; ++o) {
      float amax = 0.f;
      for (int k = 0; k < y.in; ++k) amax = std::max(amax, std::fabs(y.W[size_t(o) * y.in + k]));
      const float sw = amax > 0.f ? amax / 127.0f : 1.0f;
      h->i8_sw[l].push_back(sw);
      for (int k = 0; k < y.in; ++k) {
        float q = std::nearbyint(y.W[size_t(o) * y.in + k] / sw);
        q = std::min(127.f, std::max(-127.f, q));
        const uint32_t byte = uint32_t(int(q)) & 0xffu;
        words[w_off[l] + size_t(o) * in16[l] * 4 + k / 4] |= byte << (8 * (k % 4));
      }
    }
  }
  // device image: [scales of all layers | 127/alpha] [biases] [codes]
  size_t n_s = 0, n_b = 0;
  for (int l = 0; l < n; ++l) n_s += L[l].out, n_b += L[l].out;
  const size_t bytes = 4 * (n_s + n + n_b) + 16 + 4 * words.size();
  gnntrk_status st = alloc(h, &h->d_i8, bytes);
  if (st) return st;
  uint8_t* base = static_cast<uint8_t*>(h->d_i8);
  float* ds = reinterpret_cast<float*>(base);
  float* dinv = ds + n_s;
  float* db = dinv + n;
  uint32_t* dw = reinterpret_cast<uint32_t*>(base + ((4 * (n_s + n + n_b) + 15) / 16) * 16);
  std::vector<float> bias;
  for (int l = 0; l < n; ++l) bias.insert(bias.end(), L[l].b.begin(), L[l].b.end());
  cudaError_t e = cudaMemcpy(db, bias.data(), 4 * bias.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dw, words.data(), 4 * words.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "INT8 weight upload");
  size_t so = 0;
  for (int l = 0; l < n; ++l) {
    h->i8.l[l] = Int8Layer{dw + w_off[l], ds + so, db + so, in4[l], in16[l], L[l].out};
    so += L[l].out;
  }
  h->i8.inv = dinv;
  h->i8.n = n;
  h->i8.max_in4 = max_in4;
  return upload_i8_scales(h);
}
}  // namespace

namespace gnntrk {
// failure text of handle-less calls, returned by gnntrk_last_error(NULL)
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gnntrk

extern "C" {

void gnntrk_default_cfg(gnntrk_cfg* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_embed_layers = 3;
  c->embed_dims[0] = 3;
  c->embed_dims[1] = 64;
  c->embed_dims[2] = 64;
  c->embed_dims[3] = 4;
  c->hidden = 32;
  c->iters = 4;
  c->n_planes = 26;
  c->k_max = 64;
  c->radius2 = 1.0f;
  c->score_cut = 0.5f;
  const float fs[6] = {45.f, 3.14159265358979323846f, 750.f, 45.f, 45.f, 750.f};
  for (int i = 0; i < 6; ++i) c->feat_scale[i] = fs[i];
  c->precision = GNNTRK_FP32;
  c->rescore_band = 0.f;
  c->max_hits = 1 << 20;
  c->max_events = 4096;
  c->edges_per_hit = 24;
  c->use_graph = 0;
  c->triplets = 0;
  c->triplet_cut = 0.5f;
  c->triplets_per_hit = 16;
}

gnntrk_status gnntrk_create(const void* weights, size_t weights_bytes, const gnntrk_cfg* cfg,
                            gnntrk_handle** out) {
  if (!out) return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "cfg is NULL");
  const gnntrk_cfg& c = *cfg;
  if (c.n_embed_layers < 1 || c.n_embed_layers > kMaxEmbedLayers || c.embed_dims[0] != 3)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "embedding: 1..8 layers with 3 inputs");
  for (int l = 1; l <= c.n_embed_layers; ++l)
    if (c.embed_dims[l] < 1 || c.embed_dims[l] > 256)
      return fail(nullptr, GNNTRK_ERR_UNSUPPORTED, "embedding widths must be 1..256");
  if (!valid_d(c.embed_dims[c.n_embed_layers]))
    return fail(nullptr, GNNTRK_ERR_UNSUPPORTED, "embedding dimension must be 1..8 or 16");
  if (c.hidden != 32 && c.hidden != 64 && c.hidden != 128)
    return fail(nullptr, GNNTRK_ERR_UNSUPPORTED, "hidden must be 32, 64 or 128");
  if (c.iters < 0 || c.iters > kMaxIters)
    return fail(nullptr, GNNTRK_ERR_UNSUPPORTED, "iters must be 0..16");
  if (c.n_planes < 2 || c.n_planes > kMaxPlanes)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "n_planes must be 2..64");
  if (c.k_max < 1) return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "k_max must be >= 1");
  if (!(c.radius2 > 0.f) || !std::isfinite(c.radius2))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "radius2 must be positive and finite");
  if (!(c.score_cut > 0.f && c.score_cut < 1.f))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "score_cut must be in (0, 1)");
  for (int i = 0; i < 6; ++i)
    if (!(c.feat_scale[i] != 0.f) || !std::isfinite(c.feat_scale[i]))
      return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "feature scales must be finite and non-zero");
  if (c.precision < GNNTRK_FP32 || c.precision > GNNTRK_FP8_E4M3)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "unknown precision");
  if (c.rescore_band < 0.f || c.rescore_band >= 0.5f)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "rescore_band must be in [0, 0.5)");
  if (c.max_hits < 1 || c.max_hits > (int64_t(1) << 30))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "max_hits must be 1..2^30");
  if (c.max_events < 1 || c.max_events > 65535)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "max_events must be 1..65535");
  if (c.edges_per_hit < 1 || int64_t(c.max_hits) * c.edges_per_hit >= (int64_t(1) << 31))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "edge workspace must hold < 2^31 edges");
  if (c.triplets != 0 && c.triplets != 1)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "triplets must be 0 or 1");
  if (c.embed_int8 != 0 && c.embed_int8 != 1)
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "embed_int8 must be 0 or 1");
  if (c.triplets && !(c.triplet_cut > 0.f && c.triplet_cut < 1.f))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "triplet_cut must be in (0, 1)");
  if (c.triplets && (c.triplets_per_hit < 1 ||
                     int64_t(c.max_hits) * c.triplets_per_hit >= (int64_t(1) << 31)))
    return fail(nullptr, GNNTRK_ERR_INVALID_ARG, "triplet workspace must hold < 2^31 triplets");

  std::vector<HostLayer> L;
  std::string why;
  if (!parse_weights(weights, weights_bytes, c, L, why))
    return fail(nullptr, GNNTRK_ERR_WEIGHTS, why);

  gnntrk_handle* h = new gnntrk_handle;
  h->cfg = c;
  cudaGetDevice(&h->device);
  h->n_embed = c.n_embed_layers;
  h->D = c.embed_dims[c.n_embed_layers];
  h->h = c.hidden;
  h->K = c.iters;
  gnntrk_status st = upload_f32(h, L);
  const int n_gnn_layers = int(L.size()) - (h->has_trip ? 4 : 0);
  if (!st && c.triplets && !h->has_trip)
    st = fail(h, GNNTRK_ERR_WEIGHTS, "cfg.triplets needs a blob with the triplet classifiers");
  if (!st && c.precision != GNNTRK_FP32) st = (gnntrk_status)tc_upload(h->tc, L.data(), n_gnn_layers, h->n_embed,
                                                       h->h, h->K, c.precision, &h->d_wtc, h->err);
  if (!st && c.embed_int8) st = setup_int8(h, L);
  if (!st) st = alloc_n(h, &h->d_amax, kMaxEmbedLayers);
  for (int l = 0; l < h->n_embed; ++l) h->amax_layers.l[l] = h->embed[l];
  h->amax_layers.n = h->n_embed;
  if (!st && c.precision != GNNTRK_FP32 && c.triplets)
    st = (gnntrk_status)tc_upload_triplets(h->tc, L[n_gnn_layers], L[n_gnn_layers + 2],
                                           &h->d_wtrip, h->err);
  if (!st) st = alloc_workspace(h);
  if (!st && c.precision == GNNTRK_BF16) tc_make_maps(h->tc, h->ws, h->h);
  if (st) {
    g_create_error = h->err;
    gnntrk_destroy(h);
    return st;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cuda_fail(h, e, "create");
    g_create_error = h->err;
    gnntrk_destroy(h);
    return GNNTRK_ERR_CUDA;
  }
  *out = h;
  return GNNTRK_OK;
}

}  // extern "C"

namespace {
// One call of the path; `tracks` (when not null) adds the triplet stage.
gnntrk_status run_call(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                       const float* hits_xyz, const uint8_t* plane, const int64_t* offsets,
                       int32_t* out_labels, const TrackOut* tracks, void* stream) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  const gnntrk_cfg& c = h->cfg;
  h->want_tracks = tracks != nullptr;
  if (tracks) h->track_out = *tracks;
  const TrackOut tk = tracks ? *tracks : TrackOut{};
  if (n_events < 1 || n_events > c.max_events)
    return fail(h, GNNTRK_ERR_INVALID_ARG, "n_events out of range");
  if (n_hits < 0 || n_hits > c.max_hits) return fail(h, GNNTRK_ERR_INVALID_ARG, "n_hits out of range");
  if (n_hits > 0 && (!hits_xyz || !plane || !out_labels))
    return fail(h, GNNTRK_ERR_INVALID_ARG, "NULL input or output pointer");
  if (!offsets) return fail(h, GNNTRK_ERR_INVALID_ARG, "offsets is NULL");
  if ((reinterpret_cast<uintptr_t>(hits_xyz) & 3) || (reinterpret_cast<uintptr_t>(offsets) & 7) ||
      (reinterpret_cast<uintptr_t>(out_labels) & 3))
    return fail(h, GNNTRK_ERR_INVALID_ARG, "misaligned pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_events = n_events;
  h->last_hits = int(n_hits);
  h->last_stream = s;

  Ws& w = h->ws;
  Batch b{};
  b.n_events = n_events;
  b.n_hits = int(n_hits);
  b.x = hits_xyz;
  b.y = hits_xyz + n_hits;
  b.z = hits_xyz + 2 * n_hits;
  b.plane = plane;
  b.offsets = w.ev_off;
  b.labels = out_labels;

  if (c.use_graph && !h->profiling && s != nullptr) {
    for (auto& ge : h->graphs)
      if (ge.n_events == n_events && ge.n_hits == n_hits && ge.xyz == hits_xyz &&
          ge.plane == plane && ge.offsets == offsets && ge.labels == out_labels &&
          ge.ev_tracks == tk.ev_tracks && ge.track_off == tk.track_off &&
          ge.track_hits == tk.track_hits && ge.max_tracks == tk.max_tracks &&
          ge.max_track_hits == tk.max_hits) {
        h->last_launches = ge.launches;
        cudaError_t e = cudaGraphLaunch(ge.exec, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
        return GNNTRK_OK;
      }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream capture");
    enqueue_pipeline(h, b, offsets, s);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    if (h->graphs.size() >= 16) {
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back({n_events, n_hits, hits_xyz, plane, offsets, out_labels, tk.ev_tracks,
                         tk.track_off, tk.track_hits, tk.max_tracks, tk.max_hits, exec,
                         h->last_launches});
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    return GNNTRK_OK;
  }
  enqueue_pipeline(h, b, offsets, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "launch");
  return GNNTRK_OK;
}
}  // namespace

extern "C" {

gnntrk_status gnntrk_find_tracks(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                                 const float* hits_xyz, const uint8_t* plane,
                                 const int64_t* offsets, int32_t* out_labels, void* stream) {
  return run_call(h, n_events, n_hits, hits_xyz, plane, offsets, out_labels, nullptr, stream);
}

gnntrk_status gnntrk_find_tracks_triplets(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                                          const float* hits_xyz, const uint8_t* plane,
                                          const int64_t* offsets, int32_t* out_labels,
                                          int32_t* out_event_tracks, int64_t* out_track_off,
                                          int32_t* out_track_hits, int64_t max_tracks,
                                          int64_t max_track_hits, void* stream) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  if (!h->cfg.triplets)
    return fail(h, GNNTRK_ERR_INVALID_ARG, "the handle was created without cfg.triplets");
  if (!out_event_tracks || !out_track_off || (max_track_hits > 0 && !out_track_hits) ||
      max_tracks < 0 || max_track_hits < 0)
    return fail(h, GNNTRK_ERR_INVALID_ARG, "NULL or negative track output");
  if ((reinterpret_cast<uintptr_t>(out_event_tracks) & 3) ||
      (reinterpret_cast<uintptr_t>(out_track_off) & 7) ||
      (reinterpret_cast<uintptr_t>(out_track_hits) & 3))
    return fail(h, GNNTRK_ERR_INVALID_ARG, "misaligned pointer");
  const TrackOut t{out_event_tracks, out_track_off, out_track_hits, max_tracks, max_track_hits};
  return run_call(h, n_events, n_hits, hits_xyz, plane, offsets, out_labels, &t, stream);
}

gnntrk_status gnntrk_embed_amax(gnntrk_handle* h, int64_t n_hits, const float* hits_xyz,
                                float* out_amax, void* stream) {
  if (!h || !out_amax) return GNNTRK_ERR_INVALID_ARG;
  if (n_hits < 0 || n_hits >= (int64_t(1) << 31) || (n_hits > 0 && !hits_xyz))
    return fail(h, GNNTRK_ERR_INVALID_ARG, "n_hits out of range or NULL hits");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_embed_amax(hits_xyz, int(n_hits), h->amax_layers, graph_params(h), h->d_amax, s);
  int32_t bits[kMaxEmbedLayers];
  cudaError_t e = cudaMemcpyAsync(bits, h->d_amax, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "embedding calibration");
  for (int l = 0; l < h->n_embed; ++l) std::memcpy(&out_amax[l], &bits[l], 4);
  return GNNTRK_OK;
}

gnntrk_status gnntrk_set_embed_scales(gnntrk_handle* h, const float* alpha, int32_t n) {
  if (!h || !alpha) return GNNTRK_ERR_INVALID_ARG;
  if (!h->cfg.embed_int8) return fail(h, GNNTRK_ERR_INVALID_ARG, "the handle has no INT8 embedding");
  if (n != h->n_embed) return fail(h, GNNTRK_ERR_INVALID_ARG, "n must equal cfg.n_embed_layers");
  for (int l = 0; l < n; ++l)
    if (!(alpha[l] > 0.f) || !std::isfinite(alpha[l]))
      return fail(h, GNNTRK_ERR_INVALID_ARG, "alpha must be positive and finite");
  // the scales are read by the next launch: wait for work in flight
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  h->i8_alpha.assign(alpha, alpha + n);
  return upload_i8_scales(h);
}

gnntrk_status gnntrk_triplet_stats(gnntrk_handle* h, int64_t* out) {
  if (!h || !out) return GNNTRK_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  int32_t cnt[C_COUNT];
  e = cudaMemcpy(cnt, h->ws.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "stats read");
  const bool ran = h->want_tracks;
  out[0] = ran ? cnt[C_TRIP_A] : 0;
  out[1] = ran ? cnt[C_TRIP_E] : 0;
  out[2] = ran ? cnt[C_TRIP_KEPT] : 0;
  out[3] = ran ? cnt[C_TRACKS] : 0;
  out[4] = ran ? cnt[C_TRACK_HITS] : 0;
  out[5] = h->ws.t_cap;
  return GNNTRK_OK;
}

gnntrk_status gnntrk_get_triplets(gnntrk_handle* h, int32_t event, int64_t capacity,
                                  int32_t* type, int32_t* hits3, float* logit, uint8_t* kept,
                                  int64_t* n_triplets) {
  if (!h || !n_triplets) return GNNTRK_ERR_INVALID_ARG;
  if (!h->want_tracks) return fail(h, GNNTRK_ERR_INVALID_ARG, "the last call built no triplets");
  if (event < 0 || event >= h->last_events) return fail(h, GNNTRK_ERR_INVALID_ARG, "event out of range");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  const Ws& w = h->ws;
  int64_t off[2];
  int32_t cnt[C_COUNT];
  e = cudaMemcpy(off, w.ev_off + event, sizeof(off), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cnt, w.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "triplet read");
  if (cnt[C_STATUS] & (ST_INPUT | ST_CAPACITY))
    return fail(h, GNNTRK_ERR_CAPACITY, "the last call failed; no triplets");
  int32_t ra[2], re[2], rp[2];
  e = cudaMemcpy(&ra[0], w.trip_off_a + off[0], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ra[1], w.trip_off_a + off[1], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&re[0], w.trip_off_e + off[0], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&re[1], w.trip_off_e + off[1], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&rp[0], w.row_ptr + off[0], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&rp[1], w.row_ptr + off[1], 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "triplet read");
  const int64_t na = ra[1] - ra[0], nl = re[1] - re[0], nt = na + nl;
  *n_triplets = nt;
  if (capacity < nt) return fail(h, GNNTRK_ERR_CAPACITY, "capacity below the event's triplet count");
  const int64_t nh = off[1] - off[0], ne = rp[1] - rp[0];
  std::vector<int32_t> perm(nh), s(ne), d(ne), a1(na), a2(na), l1(nl), l2(nl);
  std::vector<uint8_t> lt(nl);
  std::vector<float> la(na), le(nl);
  std::vector<uint8_t> ka(na), kl(nl);
  auto rd = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
  };
  rd(perm.data(), w.perm + off[0], 4 * nh);
  rd(s.data(), w.src + rp[0], 4 * ne);
  rd(d.data(), w.col + rp[0], 4 * ne);
  rd(a1.data(), w.trip_a1 + ra[0], 4 * na);
  rd(a2.data(), w.trip_a2 + ra[0], 4 * na);
  rd(la.data(), w.trip_alogit + ra[0], 4 * na);
  rd(ka.data(), w.trip_akeep + ra[0], na);
  rd(l1.data(), w.trip_e1 + re[0], 4 * nl);
  rd(l2.data(), w.trip_e2 + re[0], 4 * nl);
  rd(lt.data(), w.trip_et + re[0], nl);
  rd(le.data(), w.trip_elogit + re[0], 4 * nl);
  rd(kl.data(), w.trip_ekeep + re[0], nl);
  if (e != cudaSuccess) return cuda_fail(h, e, "triplet read");
  auto loc = [&](int32_t pos) { return perm[pos - off[0]] - int32_t(off[0]); };
  auto far_src = [&](int32_t edge) { return loc(s[edge - rp[0]]); };
  auto far_dst = [&](int32_t edge) { return loc(d[edge - rp[0]]); };
  for (int64_t t = 0; t < nt; ++t) {
    int ty, A, C, B;
    float lg;
    uint8_t k;
    if (t < na) {
      ty = 0;
      A = far_src(a1[t]);
      C = far_dst(a1[t]);
      B = far_dst(a2[t]);
      lg = la[t];
      k = ka[t];
    } else {
      const int64_t u = t - na;
      ty = lt[u];
      if (ty == 1) {
        C = far_src(l1[u]);
        A = far_dst(l1[u]);
        B = far_dst(l2[u]);
      } else {
        C = far_dst(l1[u]);
        A = far_src(l1[u]);
        B = far_src(l2[u]);
      }
      lg = le[u];
      k = kl[u];
    }
    if (type) type[t] = ty;
    if (hits3) {
      hits3[3 * t] = A;
      hits3[3 * t + 1] = C;
      hits3[3 * t + 2] = B;
    }
    if (logit) logit[t] = lg;
    if (kept) kept[t] = k;
  }
  return GNNTRK_OK;
}

int64_t gnntrk_workspace_bytes(const gnntrk_cfg* c) {
  if (!c || c->max_hits < 1 || c->n_embed_layers < 1 || c->n_embed_layers > kMaxEmbedLayers ||
      c->hidden < 1 || c->iters < 0 || c->iters > kMaxIters || c->edges_per_hit < 1 ||
      c->max_events < 1)
    return 0;
  Ws w{};
  const int D = c->embed_dims[c->n_embed_layers];
  int64_t total = 0;
  for (auto& it : workspace_plan(*c, D, c->hidden, w)) total += int64_t((it.second + 255) / 256 * 256);
  // weights: the FP32 image plus, for the tensor-core paths, the packed one
  int64_t wparams = 0;
  for (int l = 0; l < c->n_embed_layers; ++l)
    wparams += int64_t(c->embed_dims[l] + 1) * ((c->embed_dims[l + 1] + 3) & ~3);
  const int64_t hh = c->hidden;
  wparams += (4 + 4 * hh) * hh + (3 * hh + 1) * hh + (hh + 1) * hh;           // encoders
  wparams += int64_t(c->iters) * 2 * ((3 * hh + 1) * hh + (hh + 1) * hh);    // steps
  wparams += (hh + 1) * hh + (hh + 1) * 4;                                   // classifier
  total += 4 * wparams;
  if (c->precision != GNNTRK_FP32) total += 2 * wparams + 64 * 1024;
  return total;
}

gnntrk_status gnntrk_autotune(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                              const float* hits_xyz, const uint8_t* plane,
                              const int64_t* offsets, int32_t* out_labels, void* stream,
                              int32_t* choice) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  if (choice)
    for (int i = 0; i < 8; ++i) choice[i] = 0;
  const bool tc = h->cfg.precision != GNNTRK_FP32;
  const int prec = h->cfg.precision, hd = h->h;
  const bool was_profiling = h->profiling;
  // time one candidate: warm-up call, then two profiled calls; stage times
  auto trial = [&](std::vector<std::pair<std::string, double>>& out) -> gnntrk_status {
    gnntrk_set_profiling(h, 0);
    gnntrk_status st = gnntrk_find_tracks(h, n_events, n_hits, hits_xyz, plane, offsets,
                                          out_labels, stream);
    if (!st) st = gnntrk_sync_status(h, stream);
    if (st) return st;
    gnntrk_set_profiling(h, 1);
    for (int r = 0; r < 2 && !st; ++r)
      st = gnntrk_find_tracks(h, n_events, n_hits, hits_xyz, plane, offsets, out_labels, stream);
    collect_stages(h);
    out.clear();
    for (auto& sa : h->stages) out.push_back({sa.name, sa.ms});
    gnntrk_set_profiling(h, 0);
    return st;
  };
  auto stage_ms = [](const std::vector<std::pair<std::string, double>>& v, const char* n) {
    for (auto& p : v)
      if (p.first == n) return p.second;
    return 1e30;
  };
  std::vector<std::pair<std::string, double>> t;
  gnntrk_status st = GNNTRK_OK;
  // 1. tensor-core kernels: resident CTAs per SM (choice[0..3])
  if (tc) {
    const char* names[4] = {"node_prep", "edge_encoder", "node_update", "edge_update"};
    double best_t[4] = {1e30, 1e30, 1e30, 1e30};
    int best_n[4] = {0, 0, 0, 0};
    for (int n = 1; n <= 8 && !st; ++n) {
      for (int f = 0; f < 4; ++f) tc_set_ctas(prec, hd, f, n);
      st = trial(t);
      for (int f = 0; f < 4; ++f) {
        const double v = stage_ms(t, names[f]);
        if (v < best_t[f]) {
          best_t[f] = v;
          best_n[f] = n;
        }
      }
    }
    for (int f = 0; f < 4; ++f) {
      tc_set_ctas(prec, hd, f, best_n[f]);
      if (choice) choice[f] = best_n[f];
    }
    // BF16 edge step at hidden 32: per-thread row copies or TMA (choice[7])
    if (!st && prec == GNNTRK_BF16 && h->tc.maps) {
      double best = 1e30;
      int best_form = 0;
      for (int form = 0; form < 3 && !st; ++form) {
        tc_set_edge_form(form);
        st = trial(t);
        const double v = stage_ms(t, "edge_update");
        if (v < best) {
          best = v;
          best_form = form;
        }
      }
      tc_set_edge_form(best_form);
      if (choice) choice[7] = best_form;
    }
  }
  // 2. FP32 kernels (the FP32 path, or the re-score of a tensor-core path):
  //    tile-shape variant per family (choice[4..6])
  const bool fp32_runs = !tc || h->cfg.rescore_band > 0.f;
  if (fp32_runs && !st) {
    const char* n32[3][2] = {{"edge_encoder", "rescore_edge_encoder"},
                             {"node_update", "rescore_node_update"},
                             {"edge_update", "rescore_edge_update"}};
    double best_t[3] = {1e30, 1e30, 1e30};
    int best_v[3] = {0, 0, 0};
    for (int v = 0; v < 3 && !st; ++v) {
      for (int f = 0; f < 3; ++f) f32_set_variant(hd, f, v);
      st = trial(t);
      for (int f = 0; f < 3; ++f) {
        const double ms = stage_ms(t, n32[f][tc ? 1 : 0]);
        if (ms < best_t[f]) {
          best_t[f] = ms;
          best_v[f] = v;
        }
      }
    }
    for (int f = 0; f < 3; ++f) {
      f32_set_variant(hd, f, best_v[f]);
      if (choice) choice[4 + f] = best_v[f];
    }
  }
  if (was_profiling) gnntrk_set_profiling(h, 1);
  // shapes captured before tuning would keep the old launch configuration
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
  return st;
}

gnntrk_status gnntrk_selftest_wait(gnntrk_handle* h, int64_t max_cycles, void* stream) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  if (max_cycles < 1 || max_cycles > 4000000000LL)
    return fail(h, GNNTRK_ERR_INVALID_ARG, "max_cycles must be 1..4e9");
  tc_wait_selftest(h->ws.counters, max_cycles, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "launch");
  return GNNTRK_OK;
}

gnntrk_status gnntrk_set_tuning(gnntrk_handle* h, const int32_t* choice) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  if (!choice) return fail(h, GNNTRK_ERR_INVALID_ARG, "choice is NULL");
  for (int f = 0; f < 4; ++f)
    if (choice[f] < 0 || choice[f] > 8)
      return fail(h, GNNTRK_ERR_INVALID_ARG, "choice[0..3] must be 0..8 CTAs per SM");
  for (int f = 4; f < 7; ++f)
    if (choice[f] < 0 || choice[f] > 2)
      return fail(h, GNNTRK_ERR_INVALID_ARG, "choice[4..6] must be an FP32 variant 0, 1 or 2");
  if (choice[7] < 0 || choice[7] > 2)
    return fail(h, GNNTRK_ERR_INVALID_ARG, "choice[7] must be an edge-step form 0, 1 or 2");
  const int prec = h->cfg.precision, hd = h->h;
  if (prec != GNNTRK_FP32)
    for (int f = 0; f < 4; ++f) tc_set_ctas(prec, hd, f, choice[f]);
  if (prec == GNNTRK_BF16) tc_set_edge_form(choice[7]);
  for (int f = 0; f < 3; ++f) f32_set_variant(hd, f, choice[4 + f]);
  // captured graphs hold the old launch configuration
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
  return GNNTRK_OK;
}

gnntrk_status gnntrk_sync_status(gnntrk_handle* h, void* stream) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  // every copy is ordered on the caller's stream (never the legacy default
  // stream, which would join the streams other threads may be capturing)
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t cnt[C_COUNT];
  cudaError_t e = cudaMemcpyAsync(cnt, h->ws.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  const int st = cnt[C_STATUS];
  if (st) {
    const int32_t zero = 0;
    e = cudaMemcpyAsync(h->ws.counters + C_STATUS, &zero, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  }
  if (st & ST_INPUT)
    return fail(h, GNNTRK_ERR_INVALID_ARG,
                "input out of range (offsets not 0..n_hits non-decreasing, or plane >= n_planes)");
  if ((st & ST_CAPACITY) && cnt[C_EDGES] <= h->ws.e_cap && h->want_tracks)
    return fail(h, GNNTRK_ERR_CAPACITY,
                "triplet stage: " + std::to_string(cnt[C_TRIP_A]) + " articulations and " +
                    std::to_string(cnt[C_TRIP_E]) + " elbows (workspace " +
                    std::to_string(h->ws.t_cap) + " each), " + std::to_string(cnt[C_TRACKS]) +
                    " tracks with " + std::to_string(cnt[C_TRACK_HITS]) + " hits (outputs " +
                    std::to_string(h->track_out.max_tracks) + ", " +
                    std::to_string(h->track_out.max_hits) + ")");
  if (st & ST_CAPACITY)
    return fail(h, GNNTRK_ERR_CAPACITY,
                "graph needs " + std::to_string(cnt[C_EDGES]) + " edges; workspace holds " +
                    std::to_string(h->ws.e_cap));
  if (st & ST_TIMEOUT) return fail(h, GNNTRK_ERR_TIMEOUT, "a bounded device wait ran out");
  if (st & ST_INTERNAL) return fail(h, GNNTRK_ERR_CUDA, "internal device check failed");
  h->err.clear();
  return GNNTRK_OK;
}

gnntrk_status gnntrk_stats(gnntrk_handle* h, int64_t* out) {
  if (!h || !out) return GNNTRK_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  int32_t cnt[C_COUNT];
  e = cudaMemcpy(cnt, h->ws.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "stats read");
  out[0] = cnt[C_EDGES];
  out[1] = cnt[C_KEPT];
  out[2] = cnt[C_BAND];
  out[3] = cnt[C_RERUN];
  out[4] = h->last_events;
  out[5] = h->last_hits;
  out[6] = h->ws.e_cap;
  out[7] = h->last_launches;
  out[8] = cnt[C_RERUN_EDGES];
  out[9] = cnt[C_RERUN_HITS];
  return GNNTRK_OK;
}

gnntrk_status gnntrk_rescore_rows(gnntrk_handle* h, int32_t n, int64_t* edges, int64_t* hits) {
  if (!h || !edges || !hits || n < 1) return GNNTRK_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) edges[i] = hits[i] = 0;
  if (h->cfg.precision == GNNTRK_FP32 || h->cfg.rescore_band <= 0.f) return GNNTRK_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  const int NL = kMaxIters + 2;
  int32_t rs[6 * NL];
  e = cudaMemcpy(rs, h->ws.rs_counts, sizeof(rs), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "re-score counts read");
  for (int i = 0; i < n && i <= h->K; ++i) {
    edges[i] = rs[2 * NL + i];
    hits[i] = rs[5 * NL + i];
  }
  return GNNTRK_OK;
}

gnntrk_status gnntrk_get_graph(gnntrk_handle* h, int32_t event, int64_t capacity, int32_t* src,
                               int32_t* dst, float* d2, float* logit, uint8_t* kept,
                               int64_t* n_edges) {
  if (!h || !n_edges) return GNNTRK_ERR_INVALID_ARG;
  if (event < 0 || event >= h->last_events) return fail(h, GNNTRK_ERR_INVALID_ARG, "event out of range");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  const Ws& w = h->ws;
  int64_t off[2];
  int32_t cnt[C_COUNT];
  e = cudaMemcpy(off, w.ev_off + event, sizeof(off), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cnt, w.counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph read");
  if (cnt[C_STATUS] & (ST_INPUT | ST_CAPACITY))
    return fail(h, GNNTRK_ERR_CAPACITY, "the last call failed; no graph");
  int32_t rp[2];
  e = cudaMemcpy(&rp[0], w.row_ptr + off[0], 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&rp[1], w.row_ptr + off[1], 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph read");
  const int64_t ne = rp[1] - rp[0];
  *n_edges = ne;
  if (capacity < ne) return fail(h, GNNTRK_ERR_CAPACITY, "capacity below the event's edge count");
  const int64_t nh = off[1] - off[0];
  std::vector<int32_t> perm(nh), s(ne), d(ne);
  e = cudaMemcpy(perm.data(), w.perm + off[0], 4 * nh, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(s.data(), w.src + rp[0], 4 * ne, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d.data(), w.col + rp[0], 4 * ne, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && d2) e = cudaMemcpy(d2, w.d2 + rp[0], 4 * ne, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && logit) e = cudaMemcpy(logit, w.logit + rp[0], 4 * ne, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && kept) e = cudaMemcpy(kept, w.keep + rp[0], ne, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph read");
  for (int64_t i = 0; i < ne; ++i) {
    if (src) src[i] = perm[s[i] - off[0]] - int32_t(off[0]);
    if (dst) dst[i] = perm[d[i] - off[0]] - int32_t(off[0]);
  }
  return GNNTRK_OK;
}

const char* gnntrk_last_error(const gnntrk_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

gnntrk_status gnntrk_set_profiling(gnntrk_handle* h, int32_t enable) {
  if (!h) return GNNTRK_ERR_INVALID_ARG;
  collect_stages(h);
  h->profiling = enable != 0;
  if (h->profiling) h->stages.clear();
  return GNNTRK_OK;
}

int32_t gnntrk_stage_times(gnntrk_handle* h, int32_t max_stages, char* names, double* total_ms,
                           int64_t* runs) {
  if (!h) return -1;
  collect_stages(h);
  const int n = int(h->stages.size());
  for (int i = 0; i < n && i < max_stages; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, h->stages[i].name.c_str(), 31);
    }
    if (total_ms) total_ms[i] = h->stages[i].ms;
    if (runs) runs[i] = h->stages[i].runs;
  }
  return n;
}

void gnntrk_destroy(gnntrk_handle* h) {
  if (!h) return;
  collect_stages(h);
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->d_wtc) cudaFree(h->d_wtc);
  if (h->d_wtrip) cudaFree(h->d_wtrip);
  delete h;
}

}  // extern "C"
