/*
 * lt.h - C ABI of the sparse lighting-matrix renderer (GB300 / sm_103a).
 *
 * Huo, Wang, Liu, Bao, "Sparse Sampling and Completion for Light Transport in
 * VPL-based Rendering".  The lighting matrix A has one row per shading point and
 * one column per VPL (or light-tree node); the image is the sum of its columns
 * (Sec. 3).  The library never forms A: it samples entries per slice in two passes
 * (Sec. 4 and 5), completes each slice at rank r and renders the image from the
 * factors (Sec. 3, step 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an lt_status.  Argument errors are reported at once.
 *   Kernels run asynchronously on the context's stream; a device-side error (a
 *   loop bound or a capacity hit inside a kernel) is latched in a device status
 *   word and returned by the next lt_sync().
 * - Every array argument is a DEVICE pointer owned by the caller (typically a
 *   PyTorch tensor) unless the name ends in _host.  The library never frees caller
 *   memory.  The context owns only its scratch memory, grown on demand and released
 *   by lt_destroy().  Base pointers of float4 planes must be 16-byte aligned.
 * - Sizes are int64_t or int32_t as declared; seeds are uint64_t.
 * - Shading points: float[3][m][4] planes  [px py pz albedo] [nx ny nz gloss]
 *   [ox oy oz 0]   (o = unit direction to the camera, gloss 0 = diffuse).
 * - VPLs: float[3][n][4] planes [px py pz albedo] [nx ny nz gloss] [ix iy iz flux]
 *   (i = unit direction back towards the light the VPL was deposited from).
 * - Occluders: float[nb][6] axis-aligned boxes [xmin ymin zmin xmax ymax zmax].
 *
 * Entry model (Sec. 3 problem statement; the paper gives no shading formula, the
 * reading is): A(i,j) = flux_j f_i(w -> w_o) f_j(w_in -> -w) G V with
 * G = max(0, n_i.w) max(0, -n_j.w) / max(d^2, d_min^2), f = albedo/pi or the
 * normalised modified Phong mix, and V the shadow-ray test of the segment between
 * the points offset by 1e-4 along their normals, restricted to t in
 * (1e-4, 1 - 1e-4), against the closed occluder boxes.  A light-tree node c acts as
 * its representative VPL scaled by I_c / I_rep(c) (Sec. 4), I = flux * albedo.
 */
#ifndef LT_H_
#define LT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lt_status;
#define LT_OK 0
#define LT_EINVAL 1      /* bad argument (null pointer, size out of range, misalignment) */
#define LT_ENOMEM 2      /* scratch allocation failed */
#define LT_ECUDA 3       /* a CUDA runtime call failed; lt_last_error() has the text */
#define LT_ELIMIT 4      /* a device loop bound or a caller capacity was reached */
#define LT_ENUMERIC 5    /* a non-finite value where a finite one was required */

typedef struct lt_ctx lt_ctx;

/* Light tree over n VPLs: 2n-1 nodes, internal nodes 0..n-2 (root 0), leaf j is
 * node n-1+j and holds VPL order[j].  All arrays device, caller-allocated. */
typedef struct {
    int64_t n;
    int32_t* order;    /* [n] VPL of leaf j (Morton order with the orientation class above) */
    int32_t* child;    /* [2n-1][2] children, -1 on leaves */
    int32_t* parent;   /* [2n-1] parent, -1 at the root */
    int32_t* range;    /* [2n-1][2] first and last leaf index covered */
    int32_t* rep;      /* [2n-1] representative VPL (child with the larger I, ties left) */
    float* I;          /* [2n-1] intensity, I_f = I_a + I_b in float32 (Sec. 4) */
    float* B;          /* [2n-1] max over the node's VPLs of f_max / albedo */
    float* aabb;       /* [2n-1][6] lo xyz, hi xyz */
} lt_tree;

/* One frame's fixed inputs: slice-ordered points, VPLs, slices, tree and the
 * global cut seen as a forest (the tree truncated at the cut). */
typedef struct {
    const float* pts;          /* [3][m][4] shading points in slice order */
    int64_t m;
    const float* vpls;         /* [3][n][4] */
    int64_t n;
    const int32_t* slice_off;  /* [S+1] rows of slice s: slice_off[s] .. slice_off[s+1]-1 */
    int32_t S;
    int32_t max_rows;          /* largest slice (host value, <= 65535) */
    lt_tree tree;
    int32_t C;                 /* global cut size (forest leaves) */
    const int32_t* forest;     /* [2C-1][8] per forest node: tree node, child0, child1, parent,
                                  first leaf, last leaf, height, 0.  Leaves 0..C-1 are the cut
                                  in leaf order; internal nodes C..2C-2 its ancestors by tree id */
    const int32_t* level_off;  /* [H+2] internal forest nodes of height h: level_nodes[level_off[h]..] */
    const int32_t* level_nodes;/* [C-1] */
    int32_t H;                 /* forest height (host value) */
    const int32_t* slice_id;   /* [S] the index each slice has in the whole frame, used in every random
                                  counter that names a slice (pass-1 rows, pass-2 draws, completion
                                  starts), or NULL for s.  A process that renders a subset of a frame's
                                  slices (the frame split over GPUs by slices) passes their indices
                                  in the whole frame and draws exactly what the whole frame draws. */
} lt_frame;

/* Per-slice sampled entries Omega_s (Sec. 4-5).  Entry keys pack (row << 16) | col
 * with row local to the slice and col an index into the slice's coarsened cut. */
typedef struct {
    int32_t* ncol;        /* [S] n'_s, columns of the coarsened cut */
    int32_t* col_node;    /* [S][C] tree node of each column, leaf order */
    float* g;             /* [S][C] column importance g = max - min of observed values (Sec. 5) */
    const int64_t* off;   /* [S+1] capacity layout: slice s owns key/val[off[s] .. off[s+1]) */
    uint32_t* key;        /* [off[S]] */
    float* val;           /* [off[S]] */
    int32_t* n1;          /* [S] pass-1 entries (first n1[s] of the slice) */
    int32_t* cnt;         /* [S] all entries (pass 1 then pass 2) */
} lt_samples;

/* Completed factors: M_s ~= U_s V_s^T at rank r (the paper's X = U, Y = V^T). */
typedef struct {
    int32_t r;            /* rank, 1..32; the row stride of U and V */
    float* U;             /* [m][r] rows in slice order */
    float* V;             /* [S][C][r] */
    int32_t* rank;        /* [S] per-slice rank r_s <= r (values clamped to 1..r), or NULL: r
                             for every slice; components r_s .. r-1 of a slice's rows are 0 */
} lt_factors;

const char* lt_status_str(lt_status s);
const char* lt_last_error(const lt_ctx* ctx);

/* Create a context on CUDA device `device`; every call of the context runs on
 * `stream`, a cudaStream_t owned by the caller (NULL = the CUDA default stream). */
lt_status lt_create(lt_ctx** ctx, int device, void* stream);
lt_status lt_destroy(lt_ctx* ctx);
/* Wait for the context's stream; return and clear the latched device status. */
lt_status lt_sync(lt_ctx* ctx);
/* Device status word (int32) that kernels latch errors into, for callers that
 * poll it themselves. */
int32_t* lt_status_word(lt_ctx* ctx);
/* Number of kernels this context has launched so far (instrumentation). */
int64_t lt_launch_count(const lt_ctx* ctx);
/* Device address and size of scratch slot `slot` of the context (debugging aid:
 * the layout of a slot is internal and may change). */
lt_status lt_debug_scratch(lt_ctx* ctx, int32_t slot, void** ptr, int64_t* bytes);
/* Cap the device scratch the context may hold: a call whose scratch would grow the
 * context's total beyond `bytes` fails with LT_ENOMEM before allocating (what the
 * context already holds stays valid).  0 removes the cap.  For hosts that give the
 * library a fixed device-memory budget, and for tests of the out-of-memory path. */
lt_status lt_set_scratch_limit(lt_ctx* ctx, int64_t bytes);

/* Occluders for the shadow rays (Sec. 6 casts rays against the scene; here a
 * uniform grid over the boxes, res^3 cells, res 0 = automatic).  The grid is built
 * on the host from a copy of the boxes and kept in the context.  nb may be 0. */
lt_status lt_scene_upload(lt_ctx* ctx, const float* boxes, int64_t nb, int32_t grid_res);

/* Triangle occluders besides the boxes (synthetic mesh scenes; the paper casts its
 * shadow rays through an SBVH over triangles, Sec. 6): tris[nt][9] (three vertices,
 * device float32) are copied into a linear BVH (Morton codes of the centroids,
 * Karras topology, bottom-up boxes); from then on every shadow test of the context
 * also tests the triangles (closed triangles, Moller-Trumbore, t in (1e-4, 1 -
 * 1e-4)).  Call after lt_scene_upload, which clears the triangles; nt = 0 clears them
 * too.  Synchronous.  LT_EINVAL while frame graphs of the context are alive. */
lt_status lt_mesh_upload(lt_ctx* ctx, const float* tris, int64_t nt);
/* Copies of the BVH for inspection (device buffers): aabb[2nt-1][6], child[nt-1][2]
 * (node ids; leaf j is node nt-1+j), leaf_tri[nt]. */
lt_status lt_mesh_bvh(const lt_ctx* ctx, float* aabb, int32_t* child, int32_t* leaf_tri);

/* Shadow test of k segments org[k][3] -> end[k][3] over t in (1e-4, 1 - 1e-4):
 * blocked[k] = 1 if a closed box or an uploaded triangle meets it (no offsets
 * applied). */
lt_status lt_shadow_test(lt_ctx* ctx, const float* org, const float* end, int64_t k,
                         uint8_t* blocked);

/* A(i, j) for `count` (point, VPL) pairs with the node factor scale[k]
 * (NULL = 1): out[k] = scale[k] * A(rows[k], vpl[k]).  Sec. 3 entry definition. */
lt_status lt_eval_pairs(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                        const int32_t* rows, const int32_t* vpl, const float* scale,
                        int64_t count, float d_min, float* out);

/* Brute force: img[i] = sum_j A(i, j) over all n VPLs (the column sum of the full
 * lighting matrix, Sec. 3; the reference images of the experiments). */
lt_status lt_bruteforce(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                        float d_min, float* img);
/* Instrumentation (no counterpart in the paper): re-runs the brute force of the same
 * points and VPLs without storing the image and returns in stats_host[4] the entries
 * (m n), the shadow rays cast (entries with a positive unoccluded value), the grid
 * cells visited and the box slab tests made.  Synchronous. */
lt_status lt_bruteforce_stats(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                              float d_min, int64_t* stats_host);

/* ---- Step 1 (Sec. 3): light tree and conservative global light cut ---------- */
/* Build the light tree of the VPLs into caller arrays sized for n. */
lt_status lt_build_tree(lt_ctx* ctx, const float* vpls, int64_t n, lt_tree* tree);
/* Global cut: test rows rows[nr] (pixel indices into pts), refinement in rounds
 * that split at most floor(growth * |cut|) nodes of error above eps, largest
 * errors first, until no node qualifies or |cut| = max_cut.  cut[max_cut] receives
 * tree node ids in leaf order, *cut_size_host its size. */
lt_status lt_build_global_cut(lt_ctx* ctx, const lt_tree* tree, const float* pts, int64_t m,
                              const float* vpls, const int32_t* rows, int64_t nr, float eps,
                              int32_t max_cut, float growth, float d_min, int32_t* cut,
                              int32_t* cut_size_host);
/* Errors of the nodes of a given cut, as one refinement round of
 * lt_build_global_cut computes them (the same kernels and summation order):
 * err[c] = max over the test rows x of bound(x, cut[c]) / estimate(x), infinite
 * where the estimate is zero and the bound is not.  cut[C] and err[C] are device
 * arrays.  Instrumentation for checking the refinement round by round. */
lt_status lt_cut_errors(lt_ctx* ctx, const lt_tree* tree, const float* pts, int64_t m, const float* vpls,
                        const int32_t* rows, int64_t nr, const int32_t* cut, int32_t C, float d_min, float* err);
/* Forest of the cut (layout in lt_frame).  forest[(2C-1)*8], level_off[max_levels+2],
 * level_nodes[C-1]; *height_host receives H. */
lt_status lt_cut_forest(lt_ctx* ctx, const lt_tree* tree, const int32_t* cut, int32_t C,
                        int32_t* forest, int32_t* level_off, int32_t max_levels,
                        int32_t* level_nodes, int32_t* height_host);

/* ---- Step 2 (Sec. 3): matrix slicing -------------------------------------- */
/* k-means of the features (p, w n) into S slices, `iters` Lloyd rounds from the
 * Morton-rank seeds; row_perm[m] lists pixels slice by slice (ascending pixel index
 * inside a slice), slice_off[S+1] delimits the slices. */
lt_status lt_make_slices(lt_ctx* ctx, const float* pts, int64_t m, int32_t S, int32_t iters,
                         float normal_weight, int32_t* row_perm, int32_t* slice_off);
/* The paper's own slicing (Sec. 6 step 2; slices of about `target` pixels, Sec. 3):
 * the 6-D vectors (p, w n) are split recursively into a binary tree.  A node of
 * n > target points splits along the feature dimension of largest extent (float32
 * extents, the first largest) at the median: the floor(n/2) points smallest in
 * (feature value, pixel index) go left keeping their order, the rest go right.
 * Leaves left to right are the slices (pixels ascending inside a slice).  The slice
 * sizes depend on m and target only: lt_split_slice_count gives their number S (a
 * host computation; -1 for bad arguments), slice_off[S+1] is written from them.
 * Synchronous (the level layout is copied from host memory). */
int32_t lt_split_slice_count(int64_t m, int32_t target);
lt_status lt_make_slices_split(lt_ctx* ctx, const float* pts, int64_t m, int32_t target, float normal_weight,
                               int32_t* row_perm, int32_t* slice_off);
/* Slices held between min_rows and max_rows rows (the uneven slices of the batched
 * workloads; no counterpart in the paper's text, which fixes the slice size only
 * roughly, Sec. 3): starting from the S slices (row_perm_in, slice_off_in, e.g. from
 * lt_make_slices), while a slice has fewer than min_rows rows and more than one is
 * left, the smallest such slice (ties: the lowest index) joins the slice whose
 * centroid is nearest to its own (float64 means of the float32 features (p, w n)
 * summed in ascending pixel order, squared Euclidean distance, ties to the lowest
 * index); then every slice of more than max_rows rows is split by the recursive 6-D
 * median split of lt_make_slices_split, its parts taking its place.  Writes
 * row_perm[m] (pixels ascending inside a slice; may be the same buffer as
 * row_perm_in), slice_off[S' + 1] and *S_out = S'.  Every slice ends inside the
 * bounds when max_rows >= 2 min_rows - 1 (a split halves).  LT_EINVAL for bad arguments, an
 * inconsistent slice_off, or S' > max_slices (S + m / floor((max_rows + 1) / 2)
 * always suffices).  Synchronous. */
lt_status lt_bound_slices(lt_ctx* ctx, const float* pts, int64_t m, const int32_t* row_perm_in,
                          const int32_t* slice_off_in, int32_t S, int32_t min_rows, int32_t max_rows,
                          float normal_weight, int32_t max_slices, int32_t* row_perm, int32_t* slice_off,
                          int32_t* S_out);
/* pts_out[3][m][4] = pts with rows permuted by row_perm. */
lt_status lt_permute_points(lt_ctx* ctx, const float* pts, int64_t m, const int32_t* row_perm,
                            float* pts_out);

/* ---- Steps 3-5 (Sec. 4, Sec. 5, Sec. 3 step 5): one frame ------------------ */
/* Pass 1 + light coarsening (Sec. 4, Eq. 2): per slice, k_c rows per cut node
 * (k_c = clamp(round(max(2, rate1 m') C I_c / I_root), 2, min(64, m')), rows
 * proportional to intensity and uniform in the slice) drawn with Philox (counter
 * t, c, slice, 1), entries evaluated, sibling pairs merged while
 * cost = eps + cost(q) < tau * S_hat.  Writes ncol, col_node, g, the pass-1
 * keys/values (n1 = cnt).  A slice whose entries exceed its capacity latches
 * LT_ELIMIT. */
lt_status lt_sample_pass1(lt_ctx* ctx, const lt_frame* f, float rate1, float tau, float d_min,
                          uint64_t seed, lt_samples* smp);
/* Pass 1 with coarsening to a target cut size instead of tau (Sec. 4, the variant
 * that orders the sibling pairs by cost and merges from the least): each slice ends
 * with min(target, C) columns when its forest allows it (a forest of several trees
 * stops at its roots).  Every sibling pair is tested (so every internal forest node
 * has its cost); the merged pairs are the C - target of smallest effective cost
 * max(cost, effective cost of the children), ties to the lower forest height and
 * then the lower forest id, which is what merging the least-cost testable pair one
 * at a time gives.  Outputs as lt_sample_pass1; LT_EINVAL for target < 1. */
lt_status lt_sample_pass1_target(lt_ctx* ctx, const lt_frame* f, float rate1, int32_t target, float d_min,
                                 uint64_t seed, lt_samples* smp);
/* Pass 2 (Sec. 5, Eq. 3): draws (column by the integer CDF of `weights` or of g when
 * weights is NULL, row uniform) with Philox (t, 0, slice, 2), keeping the first
 * ceil(rate m' n') - n1 new entries.  Appends keys (values undefined until
 * lt_eval_entries) and sets cnt. */
lt_status lt_sample_pass2(lt_ctx* ctx, const lt_frame* f, const float* weights, float rate,
                          uint64_t seed, lt_samples* smp);
/* Evaluate the entries n1[s] .. cnt[s]-1 of every slice (shadow rays inside). */
lt_status lt_eval_entries(lt_ctx* ctx, const lt_frame* f, float d_min, lt_samples* smp);
/* lt_eval_entries without any device allocation.  The paper has no counterpart:
 * this is for callers that cannot let the library allocate device memory, such as
 * a host application that owns the whole device-memory budget (a renderer plugin
 * inside a frame loop), where a cudaMalloc could fail against the fixed budget or
 * stall the device mid-frame.  Arguments, results and errors are those of
 * lt_eval_entries; the per-slice prefix it needs lives in a fixed device array of
 * the library (32 KB on every GPU that loads the library, held until exit), so
 * at most 4096 slices are accepted (LT_EINVAL beyond that).  Each call looks up
 * that array's device address (cudaGetSymbolAddress, which allocates nothing), so
 * the library keeps working after a device reset; during a stream capture the
 * lookup is not made and the address of the device's last call is used, so make
 * one call on the device before capturing (a first call inside a capture returns
 * LT_EINVAL).  All calls share the array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams or contexts) race on it and
 * must be serialised by the caller. */
lt_status lt_eval_entries_noalloc(lt_ctx* ctx, const lt_frame* f, float d_min, lt_samples* smp);
/* Instrumentation (no counterpart in the paper): re-runs the evaluation of the same
 * entries without storing values and returns in stats_host[4] the entries, the shadow
 * rays cast (entries with a positive unoccluded value), the grid cells visited and
 * the box slab tests made.  Synchronous. */
lt_status lt_eval_stats(lt_ctx* ctx, const lt_frame* f, float d_min, const lt_samples* smp,
                        int64_t* stats_host);
/* Masked ALS at rank r (uv->rank[s] per slice when given), `iters` sweeps (U-step
 * then V-step), ridge lam_rel trace(G)/r, V0 from Philox (k, j, slice, 3); float32
 * Cholesky with a float64 retry when min/max pivot^2 < 1e-6 (the retry forms the
 * line's Gram again in float64 and solves it in float64). */
lt_status lt_complete(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                      float lam_rel, uint64_t seed, lt_factors* uv);
/* Temporal coherence across frames (Sec. 7 leaves it to future work; this form is
 * ours): lt_complete started from a previous frame's factors.  Column c of slice s
 * whose coarsened-cut node (smp->col_node, a tree node id) was column i of the
 * previous frame's slice s (prev_col_node [S][C], prev_ncol [S]) starts from the
 * previous V row i (prev_V [S][C][uv->r]; its components below the slice's rank,
 * zero beyond), every other column from the seeded start of lt_complete; then
 * `iters` sweeps as lt_complete.  The previous arrays are device memory that the
 * caller keeps (prev_V must not be uv->V).  LT_EINVAL as lt_complete, or for null
 * previous arrays. */
lt_status lt_complete_warm(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                           float lam_rel, uint64_t seed, const int32_t* prev_col_node, const int32_t* prev_ncol,
                           const float* prev_V, lt_factors* uv);
/* The tensor-core contraction of one ALS half-step alone, a check of the Gram
 * matrices of the completion (Sec. 5; lt_complete with als_form 1).  Side 0: every
 * row i of every slice gets G_i = sum_j v_j v_j^T and b_i = sum_j A_ij v_j over its
 * observed entries (i, j), v_j the rows of uv->V; side 1: every column j gets the
 * same over its entries with the rows u_i of uv->U.  Written to `gram` (device,
 * float32, caller-allocated) at line L = the slice-ordered row (side 0: m lines) or
 * s C + j (side 1: S C lines), stride r (r + 3) / 2: the packed lower triangle of G
 * (element (a, c), c <= a, at a (a + 1) / 2 + c), then b.  Lines past n'_s are not
 * written.  LT_EINVAL unless 1 <= uv->r <= 16 and uv->rank is NULL. */
lt_status lt_als_gram(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_factors* uv, int32_t side,
                      float* gram);

/* Lines (rows of U or columns of V, summed over every half-step) that the last
 * lt_complete of the context solved in float64 because their float32 pivots failed
 * the check above; their Gram is formed again in float64 from the float32 factors.
 * Synchronises the context's stream.  0 before the first lt_complete.
 * Instrumentation; the paper has no counterpart. */
lt_status lt_complete_fp64_lines(lt_ctx* ctx, int64_t* count_host);
/* Nonnegative completion of every slice by the alternating direction method of
 * App. A, `iters` iterations (X step, Y step, Z, U, V, Lambda, Pi in the appendix's
 * order) at rank r (uv->rank[s] per slice when given).  Readings: the Y step uses
 * X^T Z; Lambda_{k+1} = Lambda_k + gamma alpha (X_{k+1} - U_{k+1}); P_Omega keeps
 * the observed entries (Z = M there).  Penalties alpha = alpha_rel ||Y0||_F^2 / r and
 * beta = alpha_rel ||X0||_F^2 / r from the start, constant over the iterations;
 * 0 < gamma < 1.618 (the appendix's interval).  Start: Y0^T = the lt_complete start
 * (Philox (k, j, slice, 3)), X0[i][k] = sqrt(mu / r) (0.5 + w / 2^32) with w from
 * Philox (k, i, slice, 6), mu the slice's mean observed value; U0 = X0, V0 = Y0,
 * Lambda0 = Pi0 = 0.  Writes X to uv->U ([m][r] in slice row order) and Y^T to uv->V
 * ([S][C][r]), the layout lt_render reads; a slice with no entries or mean value
 * <= 0 gets zero factors.  Float32 throughout; Z is never formed (only its observed
 * part, from the factors).  Needs device scratch of 3 m r + 2 S C r floats besides
 * the observed-entry layout.  LT_EINVAL for alpha_rel <= 0, gamma outside
 * (0, 1.618), iters < 0 or r outside 1..32. */
lt_status lt_complete_adm(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                          float alpha_rel, float gamma, uint64_t seed, lt_factors* uv);
/* Per-slice rank rule: rank[s] = min(R, max(8, 8 ceil(n'_s / cols))), a multiple of 8
 * that grows with the slice's coarsened cut (n'_s after lt_sample_pass1). */
lt_status lt_slice_ranks(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t R, int32_t cols,
                         int32_t* rank);
/* img[row_perm[slice_off[s] + i]] = max(0, u_i . (V_s^T w_s)); w NULL = all ones
 * (the column sum, Sec. 3 step 5), else w[S][C]. */
lt_status lt_render(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_factors* uv,
                    const float* w, const int32_t* row_perm, float* img);

/* ---- Colour: three channels stacked as rows of a slice --------------------
 * The paper renders coloured scenes (Sec. 6) and prints only the scalar matrix.
 * Channel k of an entry takes each factor's colour in channel k: the point's albedo
 * rho_p,k and the node intensity I_c,k = sum of the node's VPL powers
 * Phi_k rho_q,k.  An entry of the scalar frame factors as A(i, c) = rho_p(i) I_c
 * K(i, rep(c)) (K: geometry, BRDF shape, visibility; rho_p the frame's scalar
 * albedo, I_c the tree's intensity), so A_k(i, c) = A(i, c) (rho_p,k / rho_p)
 * (I_c,k / I_c): sampling runs on the scalar frame and every sampled pair gives
 * the three channels without another shadow ray.  Slice s of m' pixels becomes a
 * slice of 3m' rows, row 3i + k holding channel k of pixel i; lt_complete or
 * lt_complete_adm and lt_render then run on the stacked frame (the frame with
 * slice_off = slice_off3, m = 3m, max_rows = 3 max_rows) and write the image as
 * [m][3] through row_perm3.  All arrays device, caller-allocated. */
typedef struct {
    float* pt_ratio;      /* [m][4] rho_p,k / rho_p of slice-ordered row r (k < 3; 0 where rho_p = 0) */
    float* node_ratio;    /* [2n-1][4] I_v,k / I_v of tree node v (0 where I_v = 0) */
    int32_t* slice_off3;  /* [S+1] 3 slice_off */
    int32_t* row_perm3;   /* [3m] stacked row 3r + k -> image element 3 row_perm[r] + k */
} lt_rgb;
/* Fills `out` from pt_albedo [m][4] (RGB albedo of each pixel, image order) and
 * vpl_power [n][4] (Phi_k rho_q,k of each VPL).  LT_EINVAL when 3 max_rows > 65535
 * (stacked rows must fit the 16-bit row of a key). */
lt_status lt_rgb_setup(lt_ctx* ctx, const lt_frame* f, const float* pt_albedo, const float* vpl_power,
                       const int32_t* row_perm, lt_rgb* out);
/* Entry e of slice s (key (i, c), value v) -> entries 3e + k of the stacked slice:
 * key (3i + k, c), value v pt_ratio[row][k] node_ratio[col_node][k]; sets cnt = 3
 * cnt, n1 = 3 n1 and ncol of smp3.  smp3->off is the stacked capacity layout (3 off
 * of smp suffices); a slice beyond its capacity latches LT_ELIMIT and keeps the
 * entries that fit. */
lt_status lt_expand_rgb(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_rgb* c,
                        lt_samples* smp3);

/* ---- Launch tuning (no counterpart in the paper) ---------------------------
 * Launch shapes the library lets a caller tune per workload; they change no result
 * beyond the float rounding of the ALS Gram (als_lane_entries, als_form).  The values
 * apply to later calls and to later graph captures of the context. */
typedef struct {
    int32_t eval_ctas_per_sm;   /* entry evaluation: persistent CTAs of 128 threads per SM (1..64), 16 */
    int32_t ray_ctas_per_sm;    /* pass-1 shadow-ray kernels: the same (1..64), 16 */
    int32_t als_lane_entries;   /* ALS (r <= 16): a line gets 2^g lanes so that a lane holds at most about
                                   this many of its entries (16..1024), 96 */
    int32_t als_form;           /* ALS (r <= 16): 1 = Gram and right-hand side as dense masked products on
                                   the tensor cores (tcgen05), 0 = lane-group SIMT kernel; 0 */
    int32_t p1_form;            /* pass-1 forest levels: 1 = one persistent cooperative launch with grid-wide
                                   barriers between the steps of a level, 0 = one launch per step and
                                   level; 0 (the same results either way) */
} lt_tuning;
lt_status lt_get_tuning(const lt_ctx* ctx, lt_tuning* t);
/* LT_EINVAL (and no change) if a value is out of range. */
lt_status lt_set_tuning(lt_ctx* ctx, const lt_tuning* t);

/* ---- Learned pass-2 proposal ---------------------------------------------
 * The paper draws pass-2 columns from the pass-1 estimate g (Sec. 5) and leaves a
 * learned importance to future work; these calls are that extension.  Rows of the
 * proposal are the (slice, coarsened column) pairs, compacted: row group_off[s] + j
 * for column j < ncol[s] of slice s (group_off[S] rows in all).
 * Features (32 floats per row): mean position and mean normal of the slice's points,
 * the slice's AABB, the AABB of the column's tree node, position and normal of its
 * representative VPL, log(I_c / I_root), mean / std / log(1 + count) / min / max of
 * the column's pass-1 values (values divided by the slice's mean pass-1 value),
 * log(m') / 10 and log(n') / 10.
 * Network: 32 -> 64 -> 64 -> 64 -> 1 with SiLU; theta[LT_MLP_PARAMS] is the float32
 * master copy laid out W1[64][32] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64]
 * b4; the kernels round weights, inputs and hidden activations to bfloat16 (nearest
 * even) and accumulate in float32 on the tensor cores. */
#define LT_MLP_FEATURES 32
#define LT_MLP_HIDDEN 64
#define LT_MLP_PARAMS 10497

/* Features of every row after lt_sample_pass1: feat[S*C][32] (capacity; rows beyond
 * group_off[S] untouched), group_off[S+1] written. */
lt_status lt_proposal_features(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, float* feat,
                               int32_t* group_off);
/* Logits z[n] of the network on feat[n][32]; n = min(n_max, *n_dev) when n_dev (a
 * device int32) is given, else n_max. */
lt_status lt_proposal_forward(lt_ctx* ctx, const float* theta, const float* feat, int64_t n_max,
                              const int32_t* n_dev, float* z);
/* Pass-2 column weights w[S][C] = mix softmax_s(z)_j + (1 - mix) g_j / sum_j g_j,
 * z in row order (softmax over each slice's rows), 0 <= mix <= 1. */
lt_status lt_proposal_weights(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const int32_t* group_off,
                              const float* z, float mix, float* w);
/* Training data: the full matrix of every slice over its coarsened columns,
 * M_s[i][j] = A(row i of s, column j) row-major at M + moff[s] (moff[S+1] written);
 * a total beyond cap floats latches LT_ELIMIT and writes nothing. */
lt_status lt_slice_matrices(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, float d_min, float* M,
                            int64_t cap, int64_t* moff);
/* Training targets, in row order: p_j = (l_j + 1/n') / sum, l_j the squared norm of
 * row j of the basis after `iters` rounds of subspace iteration Q <- mgs(M^T M Q)
 * (modified Gram-Schmidt) from a Philox start (counter (k, j, slice, 4)), rank
 * min(r, n').  Slices with n' > 4096 are skipped. */
lt_status lt_leverage_targets(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const float* M,
                              const int64_t* moff, const int32_t* group_off, int32_t r, int32_t iters,
                              uint64_t seed, float* target);
/* theta = weights uniform in +-1/sqrt(fan_in) from Philox (counter (p, 0, 0, 5)), biases 0. */
lt_status lt_proposal_init(lt_ctx* ctx, uint64_t seed, float* theta);
/* Gradient grad[LT_MLP_PARAMS] of the mean over the ngroups groups (rows
 * group_off[g] .. group_off[g+1]) of the cross-entropy between target and the
 * group softmax of the logits, over n rows; the loss goes to the device float *loss
 * (may be NULL).  Deterministic (fixed reduction order). */
lt_status lt_proposal_grad(lt_ctx* ctx, const float* theta, const float* feat, const float* target,
                           const int32_t* group_off, int32_t ngroups, int64_t n, float* grad, float* loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected with `step` >= 1). */
lt_status lt_proposal_adam(lt_ctx* ctx, float* theta, float* m, float* v, const float* grad, int32_t step,
                           float lr);

/* ---- The whole frame (Sec. 3 steps 3-5) ----------------------------------- */
/* Parameters of one frame. */
typedef struct {
    float rate1;          /* pass-1 density (rows per cut node, see lt_sample_pass1) */
    float tau;            /* coarsening threshold of Eq. 2 */
    float d_min;          /* distance clamp of the geometry term */
    float rate;           /* total sampling rate of a slice (pass 1 + pass 2) */
    int32_t als_iters;    /* ALS sweeps */
    float lam_rel;        /* ALS ridge, relative to trace(G)/r */
    const float* weights; /* pass-2 column weights [S][C]; NULL = the pass-1 estimate g (Sec. 5) */
    const float* proposal;/* theta of the learned proposal; when given (and weights is NULL)
                             pass 2 draws from its weights with mixing factor `mix` */
    float mix;
    int32_t rank_cols;    /* > 0: after pass 1 the frame sets uv->rank by lt_slice_ranks with
                             R = uv->r and cols = rank_cols (uv->rank must be given); 0: fixed */
    int32_t completion;   /* LT_COMPLETE_ALS (lt_complete with als_iters, lam_rel) or
                             LT_COMPLETE_ADM (lt_complete_adm with the three values below) */
    int32_t adm_iters;
    float adm_alpha_rel;
    float adm_gamma;
    int32_t target_cut;   /* > 0: pass 1 coarsens to this many columns (lt_sample_pass1_target) */
} lt_params;
enum { LT_COMPLETE_ALS = 0, LT_COMPLETE_ADM = 1 };

/* One frame as a sequence of launches on the context's stream: lt_sample_pass1,
 * lt_sample_pass2, lt_eval_entries, lt_complete or lt_complete_adm (rank uv->r) and lt_render with
 * w = NULL, all with `seed`.  It reads two setup-dependent sizes back from the
 * device, so it synchronises the stream twice. */
lt_status lt_render_frame(lt_ctx* ctx, const lt_frame* f, const lt_params* p, uint64_t seed,
                          lt_samples* smp, lt_factors* uv, const int32_t* row_perm, float* img);

/* A frame captured once as a CUDA graph and replayed for any seed, with no host
 * synchronisation and one graph launch per frame.  The paper has no counterpart
 * (it is the batched form of the same steps).  Capture runs the frame once
 * unrecorded with seed 0 (this writes smp, uv and img), then records it; the sizes
 * read back by the unrecorded run are fixed in the graph.  The graph keeps every
 * pointer it was given (frame, samples, factors, row_perm, img, weights) and the
 * context's scene and scratch: keep them alive and unchanged in size, do not
 * re-upload the scene, and destroy the graph before the context.  Launches go to
 * the context's stream; a replay writes the same buffers as lt_render_frame with
 * the same seed.  Errors: LT_EINVAL for bad arguments, LT_ECUDA if capture or
 * instantiation fails; device errors of a replay are latched as usual. */
typedef struct lt_graph lt_graph;
lt_status lt_frame_graph_capture(lt_ctx* ctx, const lt_frame* f, const lt_params* p, lt_samples* smp,
                                 lt_factors* uv, const int32_t* row_perm, float* img, lt_graph** g);
lt_status lt_frame_graph_launch(lt_graph* g, uint64_t seed);
/* Kernels recorded in the graph (instrumentation). */
int64_t lt_frame_graph_kernels(const lt_graph* g);
lt_status lt_frame_graph_destroy(lt_graph* g);

#ifdef __cplusplus
}
#endif
#endif /* LT_H_ */
