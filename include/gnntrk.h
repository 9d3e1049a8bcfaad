/*
 * gnntrk -- GPU track finding with a graph neural network, for one GB300
 * (sm_103a). C ABI.
 *
 * The library runs, per event of a silicon-pixel vertex detector, the
 * data-parallel hot path of the ETX4VELO method (thesis "Real-Time Analysis of
 * Unstructured Data with Machine Learning on Heterogeneous Architectures",
 * chapter "ETX4VELO"):
 *
 *   1. hit embedding MLP on the normalised cylindrical (r, phi, z) of each hit
 *      (Sec. "Hit Embedding and Rough Graph Construction");
 *   2. rough graph: a hit on plane p joins hits on planes p+1 and p+2 whose
 *      squared embedding distance d^2 (Eq. of d^2) is below d^2_max, at most
 *      k_max per hit (same section, Algorithm 1);
 *   3. interaction-network GNN: node encoder on normalised (x, y, z), edge
 *      encoder on [h_i, h_j], K message-passing steps with message
 *      m_l = [sum of outgoing e, sum of incoming e] (Eq. of m^k_l) and residual
 *      node and edge networks, then the edge classifier
 *      (Sec. "Graph Neural Network and Classifiers");
 *   4. edge-score cut: edges scoring below s_edge,min are dropped, giving the
 *      purified hit graph (Sec. "The ETX4VELO Pipeline");
 *   5. weakly connected components of the purified graph as track candidates
 *      (Sec. "WCC Implementation", Algorithms 2-3).
 *
 * Conventions shared by every entry point:
 *   - Pointers named "device" are CUDA device pointers the caller owns; the
 *     library never frees or keeps them past the call (except as documented).
 *   - Pointers named "host" are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *     Device work is enqueued on it and the call returns without waiting,
 *     unless stated otherwise.
 *   - Argument errors are reported synchronously by the return value.
 *     Errors detected on the device (capacity overflow, an input out of range,
 *     a bounded wait that ran out) are latched in a status word in device
 *     memory and surface from gnntrk_sync_status(). No kernel traps.
 *   - gnntrk_last_error() returns a human-readable description of the last
 *     error of a handle (valid until the next call on that handle).
 *   - A handle is not thread safe: one host thread at a time, and calls on one
 *     handle are stream-ordered on the stream they are given. Distinct
 *     handles may be used from distinct host threads at the same time (the
 *     library's process-wide caches and tuning choices are synchronised).
 */
#ifndef GNNTRK_H
#define GNNTRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gnntrk_status {
  GNNTRK_OK = 0,
  GNNTRK_ERR_INVALID_ARG = 1, /* bad argument or input value */
  GNNTRK_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GNNTRK_ERR_OOM = 3,         /* device memory allocation failed */
  GNNTRK_ERR_CAPACITY = 4,    /* more edges than the edge workspace holds */
  GNNTRK_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  GNNTRK_ERR_WEIGHTS = 6,     /* weight blob malformed or of the wrong shape */
  GNNTRK_ERR_UNSUPPORTED = 7  /* configuration outside what is built */
} gnntrk_status;

/* Arithmetic of the MLP contractions. All of them accumulate in FP32; bias,
 * layer normalisation, residual adds, distances and the cut are FP32. */
typedef enum gnntrk_precision {
  GNNTRK_FP32 = 0,     /* FP32 operands, FP32 states (SIMT) */
  GNNTRK_BF16 = 1,     /* BF16 operands on tcgen05 tensor cores */
  GNNTRK_FP8_E4M3 = 2  /* E4M3 operands with per-output-channel weight
                          scales and per-row activation scales */
} gnntrk_precision;

/*
 * Model and run configuration.
 *
 * Model (must match the weight blob):
 *   n_embed_layers, embed_dims[0..n_embed_layers]: embedding MLP widths,
 *       embed_dims[0] = 3 (r, phi, z), embed_dims[n] = D (1..8 or 16).
 *       ReLU between layers, no activation after the last.
 *   hidden: GNN width n_h = n_e (32, 64 or 128).
 *   iters:  message-passing steps K (0..16), distinct weights per step.
 *   Every GNN sub-network is Linear -> LayerNorm (no affine, eps 1e-5) ->
 *   ReLU -> Linear.
 * Graph and cut:
 *   n_planes: detector planes (hits carry a plane id in [0, n_planes)).
 *   k_max:   maximum out-edges per hit; the k_max smallest by (d^2, plane of
 *            the target, input index of the target) are kept.
 *   radius2: d^2_max; an edge needs d^2 < radius2 (strict).
 *   score_cut: s_edge,min; an edge is kept iff sigmoid(logit) >= score_cut,
 *            evaluated as logit >= log(score_cut / (1 - score_cut)).
 *   feat_scale: divisors of the features: embedding input
 *            (r/fs[0], phi/fs[1], z/fs[2]) with phi = atan2(y, x); node
 *            encoder input (x/fs[3], y/fs[4], z/fs[5]).
 * Precision:
 *   precision: a gnntrk_precision value.
 *   rescore_band: for BF16/FP8, edges with |sigmoid(logit) - score_cut| <
 *            rescore_band are re-decided in FP32: the rows in the receptive
 *            field of those edges (per message-passing step, the hits and
 *            edges their final logit depends on; see gnntrk_rescore_rows)
 *            are recomputed in FP32 from the FP32 embedding, step by step,
 *            and only the band edges take the FP32 logit and decision.
 *            0 disables re-scoring.
 * Capacity:
 *   max_hits, max_events: largest call this handle accepts.
 *   edges_per_hit: edge workspace, in edges per hit of max_hits. A call whose
 *            graph needs more latches GNNTRK_ERR_CAPACITY (labels then invalid).
 *   use_graph: 1 = capture each call shape into a CUDA graph on first use and
 *            replay it afterwards; 0 = plain launches.
 * Triplet stage (Secs. "Triplet Building" and "Track Building"; used by
 * gnntrk_find_tracks_triplets):
 *   triplets: 1 = the handle can build tracks from triplets; the weight blob
 *            must then hold the two triplet classifiers. The last edge step
 *            then stores the final edge encodings instead of fusing the
 *            classifier.
 *   triplet_cut: triplets whose classifier score is below it are removed.
 *   triplets_per_hit: triplet workspace, per hit of max_hits, for each of
 *            the two lists (articulations, elbows); a call that needs more
 *            latches GNNTRK_ERR_CAPACITY.
 * INT8 embedding (the thesis's post-training quantisation of the embedding):
 *   embed_int8: 1 = the embedding MLP runs in INT8 in every precision: each
 *            layer's input quantised with a static scale alpha / 127
 *            (gnntrk_set_embed_scales; alpha = 1 until set, "uncalibrated"),
 *            weights per output channel (max |W_row| / 127), codes
 *            clip(round(v / S), -127, 127), INT32 dot products, then
 *            y = S_a S_w acc + b in FP32, ReLU between layers.
 */
typedef struct gnntrk_cfg {
  int32_t n_embed_layers;
  int32_t embed_dims[9];
  int32_t hidden;
  int32_t iters;
  int32_t n_planes;
  int32_t k_max;
  float radius2;
  float score_cut;
  float feat_scale[6];
  int32_t precision;
  float rescore_band;
  int64_t max_hits;
  int32_t max_events;
  int32_t edges_per_hit;
  int32_t use_graph;
  int32_t triplets;
  float triplet_cut;
  int32_t triplets_per_hit;
  int32_t embed_int8;
  int32_t reserved[3];
} gnntrk_cfg;

typedef struct gnntrk_handle gnntrk_handle;

/* Fill `cfg` with the defaults: embedding 3-64-64-4, hidden 32, 4 steps,
 * 26 planes, k_max 64, radius2 1, score cut 0.5, feature scales
 * (45, pi, 750, 45, 45, 750), FP32, no re-scoring, 1 << 20 hits, 4096 events,
 * 24 edges per hit, no CUDA graphs, no triplet stage (triplet cut 0.5,
 * 16 triplets per hit when enabled). */
void gnntrk_default_cfg(gnntrk_cfg* cfg);

/*
 * Create a handle on the current CUDA device.
 *   weights, weights_bytes: host; the weight blob (little endian):
 *     uint32 magic 0x57544E47, uint32 version 1, uint32 n_layers, uint32 0,
 *     n_layers x (uint32 fan_in, uint32 fan_out), then per layer float32
 *     W[fan_out][fan_in] followed by float32 b[fan_out]. Layer order:
 *     embedding layers; node encoder (3->h, h->h); edge encoder (2h->h, h->h);
 *     per step k: node network (3h->h, h->h), edge network (3h->h, h->h);
 *     classifier (h->h, h->1); optionally the triplet classifiers,
 *     articulation (2h->h, h->1) then elbow (2h->h, h->1), each
 *     Linear -> LayerNorm -> ReLU -> Linear on [e_first, e_second]. The blob
 *     is copied; the caller keeps ownership.
 *   cfg: host; copied.
 *   out: host; receives the handle.
 * The library allocates its device weights and workspace here and keeps them
 * until gnntrk_destroy. Errors: INVALID_ARG, WEIGHTS, UNSUPPORTED, OOM, CUDA.
 * On error *out is NULL.
 */
gnntrk_status gnntrk_create(const void* weights, size_t weights_bytes, const gnntrk_cfg* cfg,
                            gnntrk_handle** out);

/*
 * Find track candidates in a batch of events.
 *   n_events: 1..cfg.max_events.
 *   n_hits:   total hits = offsets[n_events], 0..cfg.max_hits.
 *   hits_xyz: device float32 [3][n_hits]: x (mm) at hits_xyz[0..n_hits),
 *             y at hits_xyz[n_hits..), z at hits_xyz[2 n_hits..).
 *   plane:    device uint8 [n_hits], plane id of each hit, < cfg.n_planes.
 *   offsets:  device int64 [n_events + 1]; event e owns hits
 *             [offsets[e], offsets[e+1]); offsets[0] = 0, non-decreasing.
 *   out_labels: device int32 [n_hits]; receives, for every hit, the smallest
 *             event-local input index (hit index minus offsets[e]) of its
 *             connected component in the purified graph. A track candidate
 *             is a component of at least 3 hits.
 * Hits need not be ordered by plane. Asynchronous on `stream`; the handle's
 * workspace holds the last call's graph until the next call (see
 * gnntrk_get_graph). Device-detected errors (a plane id out of range,
 * offsets inconsistent with n_hits, capacity) are latched: check them with
 * gnntrk_sync_status. Synchronous errors: INVALID_ARG, CUDA.
 */
gnntrk_status gnntrk_find_tracks(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                                 const float* hits_xyz, const uint8_t* plane,
                                 const int64_t* offsets, int32_t* out_labels, void* stream);

/*
 * Find tracks with the triplet stage (Secs. "Triplet Building" and "Track
 * Building"): the whole gnntrk_find_tracks path (its labels are written too),
 * then
 *   1. triplets of the purified graph, pairs of kept edges sharing one hit C:
 *      articulations (A->C, C->B), left elbows (C->A, C->B), right elbows
 *      (A->C, B->C); an elbow's two edges are ordered by the (plane, input
 *      index) of their far hit;
 *   2. the articulation classifier (articulations) or the elbow classifier
 *      (elbows) on [e^K(first edge), e^K(second edge)] in FP32 (the final edge
 *      encodings are FP32 or, on the tensor-core paths, BF16); a triplet is
 *      kept iff its logit >= log(c / (1 - c)) for c = cfg.triplet_cut;
 *   3. track building: kept elbows join their two edges into one group; kept
 *      articulations link groups; a link g1 -> g2 is shared when g1 links to
 *      two different groups or g2 is linked from two different groups;
 *      components of the groups over the links that are not shared; tracks
 *      are every component touching no shared link and, for every distinct
 *      pair of components (X, Y) joined by a shared link, X + Y (the shared
 *      part is duplicated into each branch); a track's hits are the endpoints
 *      of its edges, so tracks may share hits.
 * Outputs (device):
 *   out_event_tracks: int32 [n_events + 1]; event e's tracks are
 *            [out_event_tracks[e], out_event_tracks[e+1]).
 *   out_track_off: int64 [max_tracks + 1]; track t's hits are
 *            out_track_hits[out_track_off[t] .. out_track_off[t+1]).
 *   out_track_hits: int32 [max_track_hits]; event-local input indices, in
 *            (plane, index) order within a track. An event's tracks: its
 *            plain components first, then its component pairs.
 * If the tracks or their hits exceed max_tracks / max_track_hits, or the
 * triplets exceed the workspace, CAPACITY is latched (see
 * gnntrk_sync_status); gnntrk_triplet_stats then gives the sizes needed.
 * Errors: INVALID_ARG (handle without cfg.triplets, NULL or misaligned
 * outputs, the gnntrk_find_tracks argument checks), CUDA.
 */
gnntrk_status gnntrk_find_tracks_triplets(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                                          const float* hits_xyz, const uint8_t* plane,
                                          const int64_t* offsets, int32_t* out_labels,
                                          int32_t* out_event_tracks, int64_t* out_track_off,
                                          int32_t* out_track_hits, int64_t max_tracks,
                                          int64_t max_track_hits, void* stream);

/*
 * Triplet-stage counts of the last call (synchronises the device).
 *   out: host int64 [6]: [0] articulations, [1] elbows, [2] triplets kept,
 *        [3] tracks, [4] track hits (sum of track lengths), [5] triplet
 *        workspace per list. Zero when the last call had no triplet stage.
 */
gnntrk_status gnntrk_triplet_stats(gnntrk_handle* h, int64_t* out);

/*
 * Copy the triplets of one event of the last gnntrk_find_tracks_triplets
 * call to host memory (for checks; synchronises the device). Articulations
 * first, then elbows.
 *   type:  host int32 [capacity]: 0 articulation, 1 left elbow, 2 right elbow.
 *   hits3: host int32 [capacity][3]: (A, C, B) event-local input indices, C
 *          the shared hit, A the far hit of the first edge, B of the second.
 *   logit: host float32 [capacity]; kept: host uint8 [capacity].
 *   n_triplets: host; receives the event's triplet count.
 * Any of type..kept may be NULL. If capacity < *n_triplets nothing is
 * written and CAPACITY is returned.
 */
gnntrk_status gnntrk_get_triplets(gnntrk_handle* h, int32_t event, int64_t capacity,
                                  int32_t* type, int32_t* hits3, float* logit, uint8_t* kept,
                                  int64_t* n_triplets);

/*
 * Max calibration of the INT8 embedding: run the FP32 embedding over n_hits
 * hits and return, per embedding layer, the largest |input| (the first
 * layer's input is the feature vector (r/s0, phi/s1, z/s2)).
 *   hits_xyz: device float32 [3][n_hits] as for gnntrk_find_tracks.
 *   out_amax: host float [cfg.n_embed_layers].
 * Synchronises `stream`. Errors: INVALID_ARG, CUDA.
 */
gnntrk_status gnntrk_embed_amax(gnntrk_handle* h, int64_t n_hits, const float* hits_xyz,
                                float* out_amax, void* stream);

/*
 * Set the ranges alpha of the INT8 embedding's layer inputs (scale
 * alpha / 127); host float [n], n = cfg.n_embed_layers, each > 0 and
 * finite. Takes effect for the next call (also in captured CUDA graphs).
 * Errors: INVALID_ARG (no cfg.embed_int8, wrong n or value), CUDA.
 */
gnntrk_status gnntrk_set_embed_scales(gnntrk_handle* h, const float* alpha, int32_t n);

/*
 * Wait for `stream`, then return and clear the status latched by device-side
 * checks of the previous calls on this handle: OK, INVALID_ARG (input value
 * out of range), CAPACITY (edge workspace too small; labels invalid),
 * TIMEOUT (a bounded wait ran out), or CUDA (an asynchronous CUDA error).
 */
gnntrk_status gnntrk_sync_status(gnntrk_handle* h, void* stream);

/*
 * Copy the rough graph of one event of the LAST gnntrk_find_tracks call to
 * host memory (for checks and debugging; synchronises the device).
 *   event: 0..n_events-1 of that call.
 *   capacity: size of the host arrays below, in edges.
 *   src, dst: host int32 [capacity]; event-local input indices of each edge
 *             (src on the lower plane).
 *   d2:    host float32 [capacity]; squared embedding distance.
 *   logit: host float32 [capacity]; final edge logit (after any FP32
 *          re-score); score = sigmoid(logit).
 *   kept:  host uint8 [capacity]; 1 iff the edge survives the cut.
 *   n_edges: host; receives the event's edge count.
 * Any of src..kept may be NULL to skip it. If capacity < *n_edges nothing is
 * written and CAPACITY is returned (query with capacity 0).
 */
gnntrk_status gnntrk_get_graph(gnntrk_handle* h, int32_t event, int64_t capacity, int32_t* src,
                               int32_t* dst, float* d2, float* logit, uint8_t* kept,
                               int64_t* n_edges);

/*
 * Statistics of the last gnntrk_find_tracks call (synchronises the device).
 *   out: host int64 [10]: [0] total edges, [1] kept edges, [2] edges in the
 *        re-score band, [3] events holding a band edge, [4] events, [5] hits,
 *        [6] edge capacity, [7] kernels launched by the call, [8] edges and
 *        [9] hits recomputed in FP32 by the re-score (the receptive field of
 *        the band edges; 0 without a re-score).
 */
gnntrk_status gnntrk_stats(gnntrk_handle* h, int64_t* out);

/*
 * Rows recomputed by the FP32 re-score of the last gnntrk_find_tracks call,
 * per message-passing step (synchronises the device). The logit of an edge
 * after K steps of the interaction network (Sec. 3.3) depends only on its
 * K-hop neighbourhood, so the re-score evaluates, per step, only the rows in
 * the receptive field of the band edges.
 *   n:     length of both arrays (K + 1 entries are meaningful).
 *   edges: host int64 [n]: edges[0] rows of the edge encoder, edges[k + 1]
 *          rows of edge step k (edges[K] = the band edges).
 *   hits:  host int64 [n]: hits[0] rows of the node encoder, hits[k + 1] rows
 *          of node step k.
 * All zero without a re-score (FP32 precision or band 0). Errors:
 * INVALID_ARG for NULL arrays or n < 1.
 */
gnntrk_status gnntrk_rescore_rows(gnntrk_handle* h, int32_t n, int64_t* edges, int64_t* hits);

/*
 * Per-stage device timing (instrumentation for benchmarks).
 * gnntrk_set_profiling(h, 1) makes later gnntrk_find_tracks calls record a
 * CUDA event pair around each stage on the call's stream; 0 stops it. Enabling
 * also clears the accumulated times.
 * gnntrk_stage_times waits for the recorded events and reports, per stage
 * (in pipeline order), its name (NUL-terminated, at most 31 chars, written to
 * names + 32 * i), the summed device time in ms and the number of times it
 * ran. Any output may be NULL. Returns the number of stages (which may exceed
 * max_stages; only max_stages are written), or -1 on error.
 * Stage names: sort, node_prep, graph (rough graph and in-edge index),
 * edge_encoder, node_messages, node_update, edge_update, rescore_field
 * (receptive field of the band edges and its row lists), rescore_node_prep,
 * rescore_edge_encoder,
 * rescore_node_messages, rescore_node_update, rescore_edge_update,
 * components (and, for gnntrk_find_tracks_triplets, triplets,
 * triplet_scores, track_build).
 */
gnntrk_status gnntrk_set_profiling(gnntrk_handle* h, int32_t enable);
int32_t gnntrk_stage_times(gnntrk_handle* h, int32_t max_stages, char* names, double* total_ms,
                           int64_t* runs);

/*
 * Autotuner. Runs the given call repeatedly (a real call: inputs, outputs and
 * stream as for gnntrk_find_tracks) and times, per kernel family:
 *   - tensor-core kernels (BF16/FP8 handles): 1..8 resident CTAs per SM, capped
 *     by the shared memory, registers and tensor-memory columns each CTA needs;
 *     choice[0..3] = node encoder, edge encoder, node step, edge step;
 *   - FP32 SIMT kernels (FP32 handles, and the FP32 re-score of BF16/FP8 handles
 *     with a re-score band): variant 0 (4 warps per block), 1 (8 warps per
 *     block) or 2 (4 warps per block with the layer weights of the edge and
 *     node-step kernels at hidden 32 copied once per block into shared memory
 *     and the next tile's row indices loaded ahead; other kernels and widths
 *     run variant 0 then); choice[4..6] = encoders, node step, edge step;
 *   - the BF16 edge step at hidden 32 (BF16 handles): form 0 (each thread
 *     copies its row's [e, h_src, h_dst] into the tile), 1 (the tile is
 *     loaded by TMA: one box of 128 e rows and row gathers of h_src, h_dst)
 *     or 2 (TMA-loaded tiles in a ring, with a producer warp, an MMA warp and
 *     two epilogue warpgroups keeping several tiles in flight); choice[7]
 *     (0 elsewhere).
 * The fastest setting of each family is kept and applies to every handle of
 * the process with the same precision and hidden width. choice: host int32 [8]
 * or NULL. Synchronous. Errors: as gnntrk_find_tracks and
 * gnntrk_sync_status.
 */
gnntrk_status gnntrk_autotune(gnntrk_handle* h, int32_t n_events, int64_t n_hits,
                              const float* hits_xyz, const uint8_t* plane,
                              const int64_t* offsets, int32_t* out_labels, void* stream,
                              int32_t* choice);

/*
 * Applies a launch configuration without timing anything, e.g. the choice a
 * previous gnntrk_autotune returned (saved by the caller): choice[0..3] =
 * resident CTAs per SM of the tensor-core families (0 = the resource bound;
 * ignored by FP32 handles; capped by the resources each CTA needs),
 * choice[4..6] = FP32 variant 0, 1 or 2 of the encoders, node step and edge
 * step, choice[7] = BF16 edge-step form 0, 1 or 2 (used by BF16 handles at
 * hidden 32). Like the autotuner's result it applies to every
 * handle of the process with the same precision and hidden width, and drops
 * this handle's captured CUDA graphs (another handle's graphs keep the launch
 * shapes they were captured with). Results do not depend on the choice: a
 * row's arithmetic is the same in every variant. choice: host int32 [8].
 * Errors: GNNTRK_ERR_INVALID_ARG (NULL handle or choice, an entry out of
 * range; nothing is changed then). No GPU work.
 */
gnntrk_status gnntrk_set_tuning(gnntrk_handle* h, const int32_t* choice);

/*
 * Self-test of failure detection (test hook; no pipeline work). Enqueues on
 * `stream` one thread that waits on a fresh mbarrier nothing ever arrives on,
 * through the bounded wait the tensor-core kernels use, for at most
 * max_cycles SM cycles (1..4e9; about 0.5 ms per 1e6 at 2 GHz), and then
 * latches the timeout bit of the handle's device status word exactly as a
 * tensor-core kernel whose wait ran out does. The next gnntrk_sync_status on
 * that stream returns GNNTRK_ERR_TIMEOUT and clears the word; the handle stays
 * usable. Errors: GNNTRK_ERR_INVALID_ARG (NULL handle, max_cycles out of
 * range), GNNTRK_ERR_CUDA (launch).
 */
gnntrk_status gnntrk_selftest_wait(gnntrk_handle* h, int64_t max_cycles, void* stream);

/*
 * Device memory a handle created with `cfg` allocates (weights and workspace),
 * in bytes; 0 if cfg is invalid. For admission planning.
 */
int64_t gnntrk_workspace_bytes(const gnntrk_cfg* cfg);

/*
 * Serving loop with continuous batching (trigger-style request stream).
 *
 * Events arrive at given times; the server admits every event that has
 * arrived into the next batch as soon as one of its slots is free, so events
 * that arrive while others are on the GPU join the next batch instead of
 * waiting for a fixed batch to fill. Each slot has its own stream, handle
 * (resident weights and workspace) and pinned staging buffers; several batches
 * are on the device at once and their copies and kernels overlap. Slots are
 * created only while their device memory fits the budget.
 *
 *   weights, weights_bytes, model: as for gnntrk_create; the capacity fields
 *            of `model` are replaced by the batch caps below.
 *   scfg: host; n_slots (1..16, batches in flight), max_events_per_batch,
 *            max_hits_per_batch (every single event must fit; each slot's
 *            workspace is sized for it, so it sets how many slots the budget
 *            holds), memory_budget_bytes (device bytes of all slots together),
 *            apply_tuning / tuning (a saved autotuner choice applied to the
 *            slots' handles before the first batch; entries as for
 *            gnntrk_set_tuning, INVALID_ARG if one is out of range).
 *   n_events, offsets (host int64 [n_events+1]), hits_xyz (host float32
 *            [3][n_hits]), plane (host uint8 [n_hits]): the request stream,
 *            events in arrival order.
 *   arrival_s: host double [n_events], non-decreasing arrival times in
 *            seconds from the start of the run.
 *   out_labels: host int32 [n_hits]; event-local labels as gnntrk_find_tracks
 *            writes them (-1 for events of a batch that failed).
 *   done_s: host double [n_events]; time (seconds from the start) at which the
 *            event's labels were back in host memory.
 *   stats: host int64 [8] or NULL: [0] batches, [1] slots created,
 *            [2] batches that failed, [3] most batches in flight at once,
 *            [4] device bytes per slot, [5] largest batch (events),
 *            [6] wall time of the run in microseconds, [7] reserved.
 * Blocks until every event is done (the calling thread runs the loop).
 * Errors: INVALID_ARG, WEIGHTS, UNSUPPORTED, OOM (not even one slot fits the
 * budget), CUDA. gnntrk_last_error(NULL) describes them.
 */
typedef struct gnntrk_serve_cfg {
  int32_t n_slots;
  int32_t max_events_per_batch;
  int64_t max_hits_per_batch;
  int64_t memory_budget_bytes;
  int32_t apply_tuning;  /* 1: every slot applies `tuning` (gnntrk_set_tuning) */
  int32_t tuning[8];     /* a launch configuration gnntrk_autotune returned */
  int32_t reserved[7];
} gnntrk_serve_cfg;

gnntrk_status gnntrk_serve_run(const void* weights, size_t weights_bytes, const gnntrk_cfg* model,
                               const gnntrk_serve_cfg* scfg, int32_t n_events,
                               const int64_t* offsets, const float* hits_xyz,
                               const uint8_t* plane, const double* arrival_s,
                               int32_t* out_labels, double* done_s, int64_t* stats);

/*
 * Connected-component labels of one graph, WITHOUT allocating any memory.
 * The thesis has no counterpart of this call; it is here for callers that
 * cannot allocate device memory -- code running under another framework's
 * memory manager (a trigger application that hands out all device memory
 * itself and forbids allocations inside its algorithms), or a real-time path
 * that may not pay for cudaMalloc. It makes no allocation of any kind.
 *
 *   n_hits:  number of vertices, 0..GNNTRK_NOALLOC_MAX_HITS.
 *   n_edges: number of edges, 0..2^31-1.
 *   src, dst: device int32 [n_edges]; vertex indices in [0, n_hits).
 *   kept:    device uint8 [n_edges], or NULL for "all edges"; edge e joins
 *            its vertices iff kept[e] != 0.
 *   out_labels: device int32 [n_hits]; receives for each vertex the smallest
 *            vertex index of its weakly connected component. Given one event's
 *            graph from gnntrk_get_graph (src, dst, kept), these are the labels
 *            gnntrk_find_tracks wrote for that event.
 * Scratch: one fixed device array of 4 * (GNNTRK_NOALLOC_MAX_HITS + 64) bytes
 *   (4 MiB + 256 B), part of the library image: every GPU on which the library
 *   is loaded holds it until the process exits.
 * Set-up: every call looks up the array's device address with the calling
 *   thread's current device, so a call after a device reset (which may reload
 *   the library's module at another address) uses the new address. Inside a
 *   stream capture the lookup is not made; the address the last uncaptured
 *   call on that device found is used instead, so make one call on each
 *   device before capturing any, and none across a device reset.
 * Sharing: every call on a device uses the same array, which keeps the last
 *   call's contents (each call rewrites what it reads first). Calls whose work
 *   overlaps on the GPU -- on different streams or from different host threads
 *   -- race on it and give undefined labels: keep them on one stream.
 * Errors: INVALID_ARG (synchronous, nothing launched) when n_hits exceeds
 *   GNNTRK_NOALLOC_MAX_HITS, n_edges is out of range, edges are given with
 *   n_hits == 0 (no vertex can hold them) or a needed pointer is NULL; CUDA
 *   when a launch fails, or when a capture is running on a device that has
 *   had no uncaptured call yet. gnntrk_last_error(NULL) describes it.
 *   Detected on the device, with GNNTRK_OK returned: an edge index outside
 *   [0, n_hits), or a union whose bounded retries ran out (contention that
 *   does not settle); every label of that call is then -1, which no valid
 *   labelling contains.
 * Asynchronous on `stream`.
 */
#define GNNTRK_NOALLOC_MAX_HITS (1 << 20)
gnntrk_status gnntrk_components_noalloc(int64_t n_hits, int64_t n_edges, const int32_t* src,
                                        const int32_t* dst, const uint8_t* kept,
                                        int32_t* out_labels, void* stream);

/* Description of the last error on this handle ("" if none). The string is
 * owned by the handle. NULL handle: description of the calling host thread's
 * last failure of gnntrk_create, gnntrk_serve_run or
 * gnntrk_components_noalloc (valid until that thread's next such failure). */
const char* gnntrk_last_error(const gnntrk_handle* h);

/*
 * FP8-E4M3 conversion of the FP8 precision path (the symmetric quantisation
 * of the thesis's section on quantisation, with the E4M3 grid in place of
 * INT8): each value (already divided by its scale) becomes the nearest E4M3
 * code, ties to the even mantissa, saturating at +-448 (NaN -> 0x7F).
 *   in, out:   n floats in, n codes out (caller-owned).
 *   on_device: 0 -> host pointers, converted synchronously by the routine that
 *              packs FP8 weights at gnntrk_create; 1 -> device pointers,
 *              converted on `stream` (a cudaStream_t, 0 = default) by the
 *              conversion the tensor-core kernels apply to activations.
 * Errors: INVALID_ARG (n < 0, NULL pointer with n > 0), CUDA.
 */
gnntrk_status gnntrk_e4m3_encode(const float* in, uint8_t* out, int64_t n, int32_t on_device,
                                 void* stream);

/* Host: value of each E4M3 code (NaN for 0x7F and 0xFF). Errors: INVALID_ARG. */
gnntrk_status gnntrk_e4m3_decode(const uint8_t* in, float* out, int64_t n);

/*
 * Tensor-core throughput probe (a measurement for the roofline of the
 * tensor-core kernels; no pipeline work, no handle). On the current device,
 * one CTA per SM has one thread issue `iters` rounds of four tcgen05 BF16 MMAs
 * (M = 128, N = n, K = 16 each, FP32 accumulate in tensor memory, operands in
 * shared memory) back to back; *ms receives the device time of that launch
 * (synchronous; a warm-up launch runs first). Work = SMs x iters x 4 x
 * 2 x 128 x n x 16 flop.
 *   n: 32, 64, 128 or 256 (the interaction-network layers have N = hidden).
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (the bounded wait for the last MMA
 * ran out). gnntrk_last_error(NULL) describes them.
 */
gnntrk_status gnntrk_tc_throughput(int32_t n, int64_t iters, double* ms);

/* Release the handle's device memory, CUDA graphs and streams. NULL is a no-op.
 * The caller must make sure no work of this handle is still running. */
void gnntrk_destroy(gnntrk_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* GNNTRK_H */
