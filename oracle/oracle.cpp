// FP64 reference ("oracle") for the GNN track-finding hot path.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, deliberately unoptimised
// CPU restatement of what the method computes, used to check the CUDA library.
// Only the test suite, the package smoke check and the benchmark's CPU-baseline
// leg may load it. The CUDA library never calls, links or includes it, and this
// file includes nothing of the library: it has its own weight-blob reader, its
// own MLP, graph, GNN and connected-components code.
//
// Every quantity is computed in double precision from the float32 inputs and
// float32 weights (promoted exactly to double).
//
// Steps (thesis, chapter "ETX4VELO"):
//   embed       Sec. "Hit Embedding and Rough Graph Construction": an MLP maps the
//               normalised cylindrical coordinates (r, phi, z) of each hit to e_h.
//   graph       same section and Algorithm 1: a hit on plane p is joined to hits on
//               planes p+1 and p+2 whose squared embedding distance (Eq. of d^2)
//               is below d^2_max, keeping at most k_max of them per hit.
//   IN          Sec. "Graph Neural Network and Classifiers": node encoder on
//               normalised (x, y, z), edge encoder on [h_i, h_j], n message-passing
//               steps with message m_l = [sum of outgoing e, sum of incoming e]
//               (Eq. of m^k_l), residual node and edge networks with distinct
//               weights per step, then the edge classifier.
//   cut         edges whose score is below s_edge,min are dropped (purified graph).
//   components  weakly connected components of the purified graph (Algorithms 2
//               and 3, depth-first search); each component is a track candidate.
//
// Readings where the thesis is silent:
//   * features: embedding input (r/s0, phi/s1, z/s2), node-encoder input
//     (x/s3, y/s4, z/s5) with phi = atan2(y, x);
//   * every GNN sub-network (encoders, node and edge networks, classifier) is
//     Linear -> LayerNorm -> ReLU -> Linear, the layer normalisation having no
//     learnable scale or shift and eps = 1e-5 (the thesis's models used layer
//     normalisation to stabilise training, Sec. on the HLS4ML port, and its GNN
//     follows the Exa.TrkX interaction network); the embedding MLP is plain
//     Linear/ReLU with no activation after the last layer;
//   * concatenation orders: edge encoder [h_src, h_dst]; node network
//     [h, sum_out, sum_in]; edge network [e, h_src, h_dst];
//   * d^2 < d^2_max is strict; when more than k_max candidates pass, the k_max
//     smallest by the key (d^2, plane of the candidate, index of the candidate)
//     are kept;
//   * the cut keeps an edge iff its logit >= log(s/(1-s)) for the score cut s,
//     which is the same as sigmoid(logit) >= s without rounding the sigmoid;
//   * a component's label is the smallest hit index it contains.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <thread>
#include <tuple>
#include <vector>

namespace {

struct Layer {
  int in = 0, out = 0;
  std::vector<double> W;  // [out][in]
  std::vector<double> b;  // [out]
};

struct Model {
  std::vector<Layer> embed;
  Layer node_enc1, node_enc2, edge_enc1, edge_enc2;
  std::vector<Layer> node1, node2, edge1, edge2;  // per message-passing step
  Layer cls1, cls2;
  // triplet classifiers (optional): articulation and elbow, each
  // Linear(2h, h) -> LayerNorm -> ReLU -> Linear(h, 1) on [e_first, e_second]
  bool has_triplets = false;
  Layer art1, art2, elb1, elb2;
  int D = 0, h = 0, K = 0;
};

uint32_t rd_u32(const unsigned char* p) {
  return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) | (uint32_t(p[3]) << 24);
}

float rd_f32(const unsigned char* p) {
  uint32_t u = rd_u32(p);
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// out = W in + b
void linear(const Layer& L, const double* in, double* out) {
  for (int o = 0; o < L.out; ++o) {
    double acc = L.b[o];
    for (int i = 0; i < L.in; ++i) acc += L.W[size_t(o) * L.in + i] * in[i];
    out[o] = acc;
  }
}

// Layer normalisation over one vector, without learnable scale or shift:
// (v - mean) / sqrt(var + 1e-5), var the biased variance.
void layer_norm(std::vector<double>& v) {
  double mean = 0.0;
  for (double a : v) mean += a;
  mean /= double(v.size());
  double var = 0.0;
  for (double a : v) var += (a - mean) * (a - mean);
  var /= double(v.size());
  double inv = 1.0 / std::sqrt(var + 1e-5);
  for (double& a : v) a = (a - mean) * inv;
}

// GNN sub-network: Linear -> LayerNorm -> ReLU -> Linear
void mlp2(const Layer& L1, const Layer& L2, const double* in, double* out) {
  std::vector<double> t(L1.out);
  linear(L1, in, t.data());
  layer_norm(t);
  for (double& v : t) v = v > 0.0 ? v : 0.0;
  linear(L2, t.data(), out);
}

struct Params {
  int n_planes;
  int k_max;
  double r2;
  double cut_logit;
  double feat_scale[6];
};

void embed_hit(const Model& m, const Params& P, float x, float y, float z, double* e) {
  double xd = x, yd = y, zd = z;
  std::vector<double> a = {std::sqrt(xd * xd + yd * yd) / P.feat_scale[0],
                           std::atan2(yd, xd) / P.feat_scale[1], zd / P.feat_scale[2]};
  for (size_t l = 0; l < m.embed.size(); ++l) {
    std::vector<double> o(m.embed[l].out);
    linear(m.embed[l], a.data(), o.data());
    if (l + 1 < m.embed.size())
      for (double& v : o) v = v > 0.0 ? v : 0.0;
    a.swap(o);
  }
  for (int d = 0; d < m.D; ++d) e[d] = a[d];
}

double sqdist(const double* a, const double* b, int D) {
  double s = 0.0;
  for (int d = 0; d < D; ++d) s += (a[d] - b[d]) * (a[d] - b[d]);
  return s;
}

struct Edge {
  int32_t src, dst;
  double d2;
};

std::vector<Edge> rough_graph(int64_t n, const uint8_t* plane, const double* emb, int D,
                              int n_planes, double r2, int k_max) {
  std::vector<Edge> edges;
  for (int64_t i = 0; i < n; ++i) {
    int p = plane[i];
    // candidates: hits on planes p+1 and p+2 inside the squared radius
    std::vector<std::tuple<double, int, int64_t>> cand;
    for (int64_t j = 0; j < n; ++j) {
      int q = plane[j];
      if (q != p + 1 && q != p + 2) continue;
      if (q >= n_planes) continue;
      double d2 = sqdist(emb + i * D, emb + j * D, D);
      if (d2 < r2) cand.emplace_back(d2, q, j);
    }
    std::sort(cand.begin(), cand.end());
    size_t keep = std::min(cand.size(), size_t(k_max));
    for (size_t c = 0; c < keep; ++c)
      edges.push_back({int32_t(i), int32_t(std::get<2>(cand[c])), std::get<0>(cand[c])});
  }
  return edges;
}

void in_logits(const Model& m, const Params& P, int64_t n, const float* x, const float* y,
               const float* z, int64_t ne, const int32_t* src, const int32_t* dst,
               double* logit, double* e_final = nullptr) {
  const int h = m.h;
  std::vector<double> H(size_t(n) * h), E(size_t(ne) * h);
  // node encoder on normalised Cartesian coordinates
  for (int64_t l = 0; l < n; ++l) {
    double r[3] = {double(x[l]) / P.feat_scale[3], double(y[l]) / P.feat_scale[4],
                   double(z[l]) / P.feat_scale[5]};
    mlp2(m.node_enc1, m.node_enc2, r, &H[size_t(l) * h]);
  }
  // edge encoder on [h_src, h_dst]
  std::vector<double> cat(3 * h);
  for (int64_t e = 0; e < ne; ++e) {
    for (int c = 0; c < h; ++c) {
      cat[c] = H[size_t(src[e]) * h + c];
      cat[h + c] = H[size_t(dst[e]) * h + c];
    }
    mlp2(m.edge_enc1, m.edge_enc2, cat.data(), &E[size_t(e) * h]);
  }
  std::vector<double> out_sum(size_t(n) * h), in_sum(size_t(n) * h), delta(h);
  for (int k = 0; k < m.K; ++k) {
    // message: m_l = [sum over l->j of e_lj, sum over i->l of e_il]
    std::fill(out_sum.begin(), out_sum.end(), 0.0);
    std::fill(in_sum.begin(), in_sum.end(), 0.0);
    for (int64_t e = 0; e < ne; ++e)
      for (int c = 0; c < h; ++c) {
        out_sum[size_t(src[e]) * h + c] += E[size_t(e) * h + c];
        in_sum[size_t(dst[e]) * h + c] += E[size_t(e) * h + c];
      }
    // node network with residual: h <- h + N_k([h, m])
    for (int64_t l = 0; l < n; ++l) {
      for (int c = 0; c < h; ++c) {
        cat[c] = H[size_t(l) * h + c];
        cat[h + c] = out_sum[size_t(l) * h + c];
        cat[2 * h + c] = in_sum[size_t(l) * h + c];
      }
      mlp2(m.node1[k], m.node2[k], cat.data(), delta.data());
      for (int c = 0; c < h; ++c) H[size_t(l) * h + c] += delta[c];
    }
    // edge network with residual, on the updated node encodings
    for (int64_t e = 0; e < ne; ++e) {
      for (int c = 0; c < h; ++c) {
        cat[c] = E[size_t(e) * h + c];
        cat[h + c] = H[size_t(src[e]) * h + c];
        cat[2 * h + c] = H[size_t(dst[e]) * h + c];
      }
      mlp2(m.edge1[k], m.edge2[k], cat.data(), delta.data());
      for (int c = 0; c < h; ++c) E[size_t(e) * h + c] += delta[c];
    }
  }
  if (e_final) std::copy(E.begin(), E.end(), e_final);
  // edge classifier: one output unit; the sigmoid is monotone, so the logit is
  // what the cut compares
  for (int64_t e = 0; e < ne; ++e) {
    double o;
    mlp2(m.cls1, m.cls2, &E[size_t(e) * h], &o);
    logit[e] = o;
  }
}

// Weakly connected components by depth-first search (Algorithms 2 and 3), with
// an explicit stack in place of recursion. Roots are taken in increasing index
// order, so the root of each search tree is the smallest index in its component.
void components(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                const uint8_t* keep, int32_t* label) {
  std::vector<std::vector<int32_t>> adj(n);
  for (int64_t e = 0; e < ne; ++e) {
    if (keep && !keep[e]) continue;
    adj[src[e]].push_back(dst[e]);
    adj[dst[e]].push_back(src[e]);
  }
  const int32_t WHITE = -1;
  for (int64_t u = 0; u < n; ++u) label[u] = WHITE;
  std::vector<int32_t> stack;
  for (int64_t u = 0; u < n; ++u) {
    if (label[u] != WHITE) continue;
    label[u] = int32_t(u);
    stack.push_back(int32_t(u));
    while (!stack.empty()) {
      int32_t v = stack.back();
      stack.pop_back();
      for (int32_t w : adj[v])
        if (label[w] == WHITE) {
          label[w] = int32_t(u);
          stack.push_back(w);
        }
    }
  }
}

struct EventOut {
  std::vector<Edge> edges;
  std::vector<double> logit;
  std::vector<uint8_t> keep;
};

void find_tracks_event(const Model& m, const Params& P, int64_t n, const float* x,
                       const float* y, const float* z, const uint8_t* plane, int32_t* labels,
                       EventOut* out) {
  std::vector<double> emb(size_t(n) * m.D);
  for (int64_t i = 0; i < n; ++i) embed_hit(m, P, x[i], y[i], z[i], &emb[size_t(i) * m.D]);
  std::vector<Edge> edges = rough_graph(n, plane, emb.data(), m.D, P.n_planes, P.r2, P.k_max);
  int64_t ne = int64_t(edges.size());
  std::vector<int32_t> s(ne), d(ne);
  for (int64_t e = 0; e < ne; ++e) {
    s[e] = edges[e].src;
    d[e] = edges[e].dst;
  }
  std::vector<double> logit(ne);
  in_logits(m, P, n, x, y, z, ne, s.data(), d.data(), logit.data());
  std::vector<uint8_t> keep(ne);
  for (int64_t e = 0; e < ne; ++e) keep[e] = logit[e] >= P.cut_logit ? 1 : 0;
  components(n, ne, s.data(), d.data(), keep.data(), labels);
  if (out) {
    out->edges.swap(edges);
    out->logit.swap(logit);
    out->keep.swap(keep);
  }
}

Params make_params(int n_planes, int k_max, double r2, double cut_logit, const double* fs) {
  Params P;
  P.n_planes = n_planes;
  P.k_max = k_max;
  P.r2 = r2;
  P.cut_logit = cut_logit;
  for (int i = 0; i < 6; ++i) P.feat_scale[i] = fs[i];
  return P;
}

}  // namespace

extern "C" {

// Parse a weight blob (magic "GNTW", version 1) and check it against the
// expected architecture. Returns nullptr and fills `err` on any mismatch.
void* orc_model_load(const void* blob, size_t nbytes, int n_embed_layers, const int* embed_dims,
                     int hidden, int iters, char* err, int errlen) {
  auto fail = [&](const char* msg) -> void* {
    if (err && errlen > 0) std::snprintf(err, size_t(errlen), "%s", msg);
    return nullptr;
  };
  const unsigned char* p = static_cast<const unsigned char*>(blob);
  if (nbytes < 16) return fail("blob too short");
  if (rd_u32(p) != 0x57544E47u) return fail("bad magic");
  if (rd_u32(p + 4) != 1u) return fail("bad version");
  uint32_t nl = rd_u32(p + 8);
  std::vector<std::pair<int, int>> want;
  for (int l = 0; l < n_embed_layers; ++l) want.push_back({embed_dims[l], embed_dims[l + 1]});
  const int h = hidden;
  want.push_back({3, h});
  want.push_back({h, h});
  want.push_back({2 * h, h});
  want.push_back({h, h});
  for (int k = 0; k < iters; ++k) {
    want.push_back({3 * h, h});
    want.push_back({h, h});
    want.push_back({3 * h, h});
    want.push_back({h, h});
  }
  want.push_back({h, h});
  want.push_back({h, 1});
  // optional triplet classifiers: articulation then elbow
  const bool trip = nl == want.size() + 4;
  if (trip)
    for (int t = 0; t < 2; ++t) {
      want.push_back({2 * h, h});
      want.push_back({h, 1});
    }
  if (nl != want.size()) return fail("layer count does not match the architecture");
  if (nbytes < 16 + 8 * size_t(nl)) return fail("blob too short for its header");
  std::vector<Layer> L(nl);
  size_t need = 16 + 8 * size_t(nl);
  for (uint32_t l = 0; l < nl; ++l) {
    L[l].in = int(rd_u32(p + 16 + 8 * l));
    L[l].out = int(rd_u32(p + 20 + 8 * l));
    if (L[l].in != want[l].first || L[l].out != want[l].second)
      return fail("layer shape does not match the architecture");
    need += 4 * (size_t(L[l].in) * L[l].out + L[l].out);
  }
  if (nbytes != need) return fail("blob size does not match its header");
  size_t off = 16 + 8 * size_t(nl);
  for (uint32_t l = 0; l < nl; ++l) {
    L[l].W.resize(size_t(L[l].in) * L[l].out);
    L[l].b.resize(L[l].out);
    for (auto& w : L[l].W) {
      w = rd_f32(p + off);
      off += 4;
    }
    for (auto& b : L[l].b) {
      b = rd_f32(p + off);
      off += 4;
    }
  }
  Model* m = new Model;
  size_t c = 0;
  for (int l = 0; l < n_embed_layers; ++l) m->embed.push_back(L[c++]);
  m->node_enc1 = L[c++];
  m->node_enc2 = L[c++];
  m->edge_enc1 = L[c++];
  m->edge_enc2 = L[c++];
  for (int k = 0; k < iters; ++k) {
    m->node1.push_back(L[c++]);
    m->node2.push_back(L[c++]);
    m->edge1.push_back(L[c++]);
    m->edge2.push_back(L[c++]);
  }
  m->cls1 = L[c++];
  m->cls2 = L[c++];
  if (trip) {
    m->has_triplets = true;
    m->art1 = L[c++];
    m->art2 = L[c++];
    m->elb1 = L[c++];
    m->elb2 = L[c++];
  }
  m->D = embed_dims[n_embed_layers];
  m->h = hidden;
  m->K = iters;
  return m;
}

void orc_model_free(void* m) { delete static_cast<Model*>(m); }

int orc_embed(const void* mp, int64_t n, const float* x, const float* y, const float* z,
              const double* feat_scale, double* emb) {
  const Model& m = *static_cast<const Model*>(mp);
  Params P = make_params(0, 0, 0.0, 0.0, feat_scale);
  for (int64_t i = 0; i < n; ++i) embed_hit(m, P, x[i], y[i], z[i], emb + i * m.D);
  return 0;
}

// Rough graph of one event. Returns the edge count; if it exceeds `cap`, only
// the count is returned and nothing is written.
int64_t orc_radius_graph(int64_t n, const uint8_t* plane, const double* emb, int D,
                         int n_planes, double r2, int k_max, int32_t* src, int32_t* dst,
                         double* d2, int64_t cap) {
  std::vector<Edge> e = rough_graph(n, plane, emb, D, n_planes, r2, k_max);
  int64_t ne = int64_t(e.size());
  if (ne <= cap)
    for (int64_t i = 0; i < ne; ++i) {
      src[i] = e[i].src;
      dst[i] = e[i].dst;
      d2[i] = e[i].d2;
    }
  return ne;
}

int orc_in_logits(const void* mp, int64_t n, const float* x, const float* y, const float* z,
                  const double* feat_scale, int64_t ne, const int32_t* src, const int32_t* dst,
                  double* logit) {
  const Model& m = *static_cast<const Model*>(mp);
  Params P = make_params(0, 0, 0.0, 0.0, feat_scale);
  in_logits(m, P, n, x, y, z, ne, src, dst, logit);
  return 0;
}

int orc_components(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                   const uint8_t* keep, int32_t* labels) {
  components(n, ne, src, dst, keep, labels);
  return 0;
}

// Whole hot path for one event. Labels are always written. Edge outputs are
// written when `cap` is large enough; the edge count is returned either way.
int64_t orc_find_tracks_event(const void* mp, int n_planes, int k_max, double r2,
                              double cut_logit, const double* feat_scale, int64_t n,
                              const float* x, const float* y, const float* z,
                              const uint8_t* plane, int32_t* labels, int32_t* src, int32_t* dst,
                              double* d2, double* logit, uint8_t* keep, int64_t cap) {
  const Model& m = *static_cast<const Model*>(mp);
  Params P = make_params(n_planes, k_max, r2, cut_logit, feat_scale);
  EventOut out;
  find_tracks_event(m, P, n, x, y, z, plane, labels, &out);
  int64_t ne = int64_t(out.edges.size());
  if (ne <= cap)
    for (int64_t e = 0; e < ne; ++e) {
      src[e] = out.edges[e].src;
      dst[e] = out.edges[e].dst;
      d2[e] = out.edges[e].d2;
      logit[e] = out.logit[e];
      keep[e] = out.keep[e];
    }
  return ne;
}

// Many events, one event per worker thread at a time (events are independent).
// Labels are event-local. Returns the total edge count.
int64_t orc_find_tracks_batch(const void* mp, int n_planes, int k_max, double r2,
                              double cut_logit, const double* feat_scale, int n_events,
                              const int64_t* offsets, const float* x, const float* y,
                              const float* z, const uint8_t* plane, int32_t* labels,
                              int threads) {
  const Model& m = *static_cast<const Model*>(mp);
  Params P = make_params(n_planes, k_max, r2, cut_logit, feat_scale);
  if (threads < 1) threads = 1;
  std::vector<int64_t> edges(threads, 0);
  auto work = [&](int t) {
    for (int ev = t; ev < n_events; ev += threads) {
      int64_t a = offsets[ev], b = offsets[ev + 1];
      EventOut out;
      find_tracks_event(m, P, b - a, x + a, y + a, z + a, plane + a, labels + a, &out);
      edges[t] += int64_t(out.edges.size());
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
  int64_t tot = 0;
  for (int64_t e : edges) tot += e;
  return tot;
}

// ---------------------------------------------------------------------------
// Triplet stage (Secs. "Triplet Building" and "Track Building")
// ---------------------------------------------------------------------------

// Final edge encodings e^K [ne][h] of the interaction network (the input of
// the edge and triplet classifiers).
int orc_edge_states(const void* mp, int64_t n, const float* x, const float* y, const float* z,
                    const double* feat_scale, int64_t ne, const int32_t* src, const int32_t* dst,
                    double* e_final) {
  const Model& m = *static_cast<const Model*>(mp);
  Params P = make_params(0, 0, 0.0, 0.0, feat_scale);
  std::vector<double> logit(ne);
  in_logits(m, P, n, x, y, z, ne, src, dst, logit.data(), e_final);
  return 0;
}

// Triplets of the purified graph: pairs of kept edges sharing one hit C.
//   type 0, articulation: A -> C and C -> B     (e1 = A->C, e2 = C->B)
//   type 1, left elbow:   C -> A and C -> B     (e1 = C->A, e2 = C->B)
//   type 2, right elbow:  A -> C and B -> C     (e1 = A->C, e2 = B->C)
// An elbow's two edges are ordered by the (plane, index) of their far hit,
// A before B. Triplets are listed by C ascending, then type, then the far
// hits' keys. Returns the count; writes only when it fits `cap`.
int64_t orc_triplets(int64_t n, const uint8_t* plane, int64_t ne, const int32_t* src,
                     const int32_t* dst, const uint8_t* keep, int32_t* type, int32_t* e1,
                     int32_t* e2, int64_t cap) {
  std::vector<std::vector<int32_t>> in(n), out(n);
  for (int64_t e = 0; e < ne; ++e) {
    if (!keep[e]) continue;
    out[src[e]].push_back(int32_t(e));
    in[dst[e]].push_back(int32_t(e));
  }
  // far-hit key of an edge seen from C
  auto key = [&](int32_t far) { return std::make_pair(int(plane[far]), far); };
  auto by_dst = [&](int32_t a, int32_t b) { return key(dst[a]) < key(dst[b]); };
  auto by_src = [&](int32_t a, int32_t b) { return key(src[a]) < key(src[b]); };
  int64_t t = 0;
  auto put = [&](int ty, int32_t a, int32_t b) {
    if (t < cap) {
      type[t] = ty;
      e1[t] = a;
      e2[t] = b;
    }
    ++t;
  };
  for (int64_t c = 0; c < n; ++c) {
    std::vector<int32_t> I = in[c], O = out[c];
    std::sort(I.begin(), I.end(), by_src);
    std::sort(O.begin(), O.end(), by_dst);
    for (int32_t a : I)
      for (int32_t b : O) put(0, a, b);
    for (size_t i = 0; i < O.size(); ++i)
      for (size_t j = i + 1; j < O.size(); ++j) put(1, O[i], O[j]);
    for (size_t i = 0; i < I.size(); ++i)
      for (size_t j = i + 1; j < I.size(); ++j) put(2, I[i], I[j]);
  }
  return t;
}

// Triplet logits: the articulation classifier for type 0, the elbow
// classifier for types 1 and 2, on [e^K(e1), e^K(e2)].
int orc_triplet_logits(const void* mp, int64_t nt, const int32_t* type, const int32_t* e1,
                       const int32_t* e2, const double* e_final, double* logit) {
  const Model& m = *static_cast<const Model*>(mp);
  if (!m.has_triplets) return -1;
  const int h = m.h;
  std::vector<double> cat(2 * h);
  for (int64_t t = 0; t < nt; ++t) {
    for (int c = 0; c < h; ++c) {
      cat[c] = e_final[size_t(e1[t]) * h + c];
      cat[h + c] = e_final[size_t(e2[t]) * h + c];
    }
    const bool art = type[t] == 0;
    mlp2(art ? m.art1 : m.elb1, art ? m.art2 : m.elb2, cat.data(), &logit[t]);
  }
  return 0;
}

namespace {
struct Dsu {
  std::vector<int64_t> p;
  explicit Dsu(int64_t n) : p(n) {
    for (int64_t i = 0; i < n; ++i) p[i] = i;
  }
  int64_t find(int64_t a) {
    while (p[a] != a) a = p[a] = p[p[a]];
    return a;
  }
  void unite(int64_t a, int64_t b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};
}  // namespace

// Track building from the purified edge graph, in the thesis's four steps:
//  1. kept elbows join their two edges into one group (the two edges are the
//     same track segment; the second one is the duplicate);
//  2. kept articulations link groups, once per ordered group pair; a link
//     g1 -> g2 is shared when g1 links onwards to more than one group or g2
//     is reached from more than one group; weakly connected components of the
//     groups over the links that are not shared;
//  3. every component touching no shared link is a track; every distinct pair
//     of components (X, Y) joined by a shared link X -> Y is a track X + Y
//     (the shared component is duplicated into each branch);
//  4. a track's hits are the endpoints of its edges.
// Tracks are written with their hits ascending, in lexicographic order of
// the hit lists. Returns the track count and sets *total_hits; writes only
// when both fit (track_off[tracks + 1], track_hits[total_hits]).
int64_t orc_build_tracks(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                         const uint8_t* keep, int64_t nt, const int32_t* type, const int32_t* e1,
                         const int32_t* e2, const uint8_t* tkeep, int32_t* track_off,
                         int64_t cap_tracks, int32_t* track_hits, int64_t cap_hits,
                         int64_t* total_hits) {
  (void)n;
  Dsu grp(ne);
  for (int64_t t = 0; t < nt; ++t)
    if (tkeep[t] && type[t] != 0) grp.unite(e1[t], e2[t]);
  std::vector<std::pair<int64_t, int64_t>> links;
  for (int64_t t = 0; t < nt; ++t)
    if (tkeep[t] && type[t] == 0) {
      const int64_t a = grp.find(e1[t]), b = grp.find(e2[t]);
      if (a != b) links.push_back({a, b});
    }
  std::sort(links.begin(), links.end());
  links.erase(std::unique(links.begin(), links.end()), links.end());
  std::vector<int> n_out(ne, 0), n_in(ne, 0);
  for (auto& l : links) {
    ++n_out[l.first];
    ++n_in[l.second];
  }
  Dsu comp(ne);
  std::vector<std::pair<int64_t, int64_t>> shared;
  for (auto& l : links) {
    if (n_out[l.first] > 1 || n_in[l.second] > 1)
      shared.push_back(l);
    else
      comp.unite(l.first, l.second);
  }
  // hits of every component of kept edges
  std::vector<std::vector<int32_t>> hits(ne);
  for (int64_t e = 0; e < ne; ++e) {
    if (!keep[e]) continue;
    const int64_t c = comp.find(grp.find(e));
    hits[c].push_back(src[e]);
    hits[c].push_back(dst[e]);
  }
  std::vector<std::pair<int64_t, int64_t>> pairs;
  std::vector<char> in_shared(ne, 0);
  for (auto& l : shared) {
    const int64_t a = comp.find(l.first), b = comp.find(l.second);
    if (a == b) continue;
    pairs.push_back({a, b});
    in_shared[a] = in_shared[b] = 1;
  }
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  std::vector<std::vector<int32_t>> tracks;
  auto uniq = [](std::vector<int32_t> v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
  };
  for (int64_t c = 0; c < ne; ++c)
    if (!hits[c].empty() && !in_shared[c]) tracks.push_back(uniq(hits[c]));
  for (auto& pr : pairs) {
    std::vector<int32_t> v = hits[pr.first];
    v.insert(v.end(), hits[pr.second].begin(), hits[pr.second].end());
    tracks.push_back(uniq(v));
  }
  std::sort(tracks.begin(), tracks.end());
  int64_t th = 0;
  for (auto& t : tracks) th += int64_t(t.size());
  *total_hits = th;
  const int64_t nk = int64_t(tracks.size());
  if (track_off && nk <= cap_tracks && th <= cap_hits) {
    int64_t o = 0;
    track_off[0] = 0;
    for (int64_t k = 0; k < nk; ++k) {
      for (int32_t v : tracks[k]) track_hits[o++] = v;
      track_off[k + 1] = int32_t(o);
    }
  }
  return nk;
}

// All candidate pairs (plane p to p+1 or p+2) with their squared distance, no
// radius and no cap; used to pick the squared radius that gives a mean degree.
int64_t orc_candidate_d2(int64_t n, const uint8_t* plane, const double* emb, int D,
                         int n_planes, double* out, int64_t cap) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int p = plane[i], q = plane[j];
      if ((q == p + 1 || q == p + 2) && q < n_planes) {
        if (c < cap) out[c] = sqdist(emb + i * D, emb + j * D, D);
        ++c;
      }
    }
  return c;
}

}  // extern "C"
