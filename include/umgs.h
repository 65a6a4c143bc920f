/*
 * umgs.h - C ABI of libumgs: single-pass anti-aliased rasterization of
 * triangle meshes and 3D Gaussians, and Gaussian-centric proxy-mesh binding
 * and deformation (UniMGS, arXiv 2601.19233), as hand-written CUDA kernels
 * for GB300 (sm_103a).
 *
 * General rules
 *  - Every array argument is a DEVICE pointer on the context's device, owned
 *    by the caller, unless the comment says "host".  Output arrays are
 *    allocated by the caller.  Structs describing cameras are host values.
 *  - All float arrays are IEEE binary32, row-major, densely packed.
 *  - Calls are asynchronous on the given CUDA stream (cudaStream_t passed as
 *    void*; NULL = the legacy default stream) unless the comment says that
 *    the call synchronises.
 *  - No call aborts, traps or exits.  Every call returns a umgs_status; on
 *    failure umgs_last_error(ctx) returns a message valid until the next call
 *    on the same context.  A context must not be used by two host threads at
 *    the same time.
 *  - Workspace (projected records, keys, saved state) is owned by the context
 *    or by a umgs_frame and grows on demand with cudaMalloc.
 */
#ifndef UMGS_H
#define UMGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UMGS_OK = 0,
    UMGS_ERR_INVALID_ARG = 1,     /* bad pointer, size, mode or camera */
    UMGS_ERR_OUT_OF_MEMORY = 2,   /* workspace allocation failed */
    UMGS_ERR_CAPACITY = 3,        /* a fixed-capacity device buffer overflowed */
    UMGS_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed */
    UMGS_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up */
    UMGS_ERR_NOT_IMPLEMENTED = 6
} umgs_status;

/* blend modes (Sec. 3.2, Fig. 3 / Fig. 4) */
enum {
    UMGS_BLEND_FULL = 0,        /* depth-adjacent triangle entities with 4-sample t^j (Eq. 7-9) */
    UMGS_BLEND_DIRECT = 1,      /* triangles as plain fragments, centre coverage (Fig. 3a) */
    UMGS_BLEND_MSAA_ALL = 2,    /* Eq. 5-6: pixel-level T, O_i = mean coverage (Fig. 3b) */
    UMGS_BLEND_ENTITY_ALL = 3   /* one entity across Gaussians: colour overflow (Fig. 3c) */
};

/* SH coefficient storage */
enum { UMGS_F32 = 0, UMGS_BF16 = 1 };

/* binding modes (Sec. 3.3) */
enum { UMGS_BIND_BBX = 0, UMGS_BIND_CENTER = 1, UMGS_BIND_NEAREST = 2 };

/* deformation modes: the mean update of Eq. 13 (FRAME or LITERAL), optionally
 * OR'ed with ONE_RING for the per-vertex transform (see umgs_deform) */
enum { UMGS_DEFORM_FRAME = 0, UMGS_DEFORM_LITERAL = 1, UMGS_DEFORM_ONE_RING = 16 };

typedef struct umgs_ctx umgs_ctx;
typedef struct umgs_frame umgs_frame;

/* Gaussians (Sec. 3.3: mean mu, covariance Sigma; colour from SH as in 3DGS). */
typedef struct {
    const float* means;      /* [n,3] */
    const float* quats;      /* [n,4] (w,x,y,z); normalised inside; ignored when cov3d != NULL */
    const float* scales;     /* [n,3] activated standard deviations; ignored when cov3d != NULL */
    const float* opacities;  /* [n] activated opacity in [0,1] */
    const void* sh;          /* [n,(sh_degree+1)^2,3] float32 or bfloat16 (sh_dtype); 16-byte aligned
                                when a row's bytes are a multiple of 16 (float32 degree 1 and 3,
                                bfloat16 degree 3), 8-byte aligned for bfloat16 degree 1 */
    const float* cov3d;      /* nullable [n,6] (xx,xy,xz,yy,yz,zz), e.g. the output of umgs_deform */
    int64_t n;
    int32_t sh_degree;       /* 0..3 */
    int32_t sh_dtype;        /* UMGS_F32 or UMGS_BF16 */
} umgs_gaussians;

/* A triangle mesh with per-vertex colour and alpha (Sec. 3.2: c_i, alpha_i),
 * or a textured mesh: with uv and texture given, c_i at a pixel is the
 * bilinear (clamp-to-edge) texture value at the perspective-correct
 * interpolation of the vertex uv (texel (i, j) centred at ((i+0.5)/tex_w,
 * (j+0.5)/tex_h)); vcolor is then unused and may be NULL.  Textured meshes
 * render in every mode but have no backward (NOT_IMPLEMENTED). */
typedef struct {
    const float* verts;      /* [nv,3] world positions */
    const int32_t* faces;    /* [nf,3] vertex indices in [0,nv) */
    const float* vcolor;     /* [nv,3] linear RGB (NULL allowed for a textured mesh) */
    const float* valpha;     /* nullable [nv] per-vertex alpha, interpolated */
    const float* falpha;     /* nullable [nf] per-face alpha, overrides valpha */
    int64_t nv, nf;
    const float* uv;         /* nullable [nv,2] texture coordinates */
    const float* texture;    /* nullable [tex_h,tex_w,3] linear RGB, row-major (with uv) */
    int32_t tex_w, tex_h;
} umgs_mesh;

/* Pinhole camera, world->camera [R|t], x right, y down, z forward;
 * pixel (x,y) has its centre at (x+0.5, y+0.5); u = fx*X/Z + cx. */
typedef struct {
    float viewmat[12];       /* row-major 3x4 [R|t] */
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;            /* primitives with Z <= near_z are culled */
} umgs_camera;

/* umgs_render_opts.flags */
enum {
    UMGS_RENDER_SAVE_BACKWARD = 1,  /* keep per-pixel state for umgs_render_backward (FULL mode) */
    UMGS_RENDER_MIXED = 2,          /* Gaussian fragment records in fp16 (screen position fp32), fp32
                                       blending; pair with bf16 SH for the mixed-precision form.  Keys,
                                       footprints and order are unchanged (still exact); no backward. */
    UMGS_RENDER_T_PRODUCT = 4,      /* FULL mode only: inside an entity T <- T (1 - O_i alpha_i), the
                                       literal reading of Sec. 3.2's Eq. 6 instead of T = T_in mean_j t^j
                                       (the two agree for one-triangle entities); no backward. */
    UMGS_RENDER_ASYNC = 8,          /* no host read-back inside umgs_render: the (tile, primitive) pairs
                                       are held to the frame's reserved capacity (umgs_frame_reserve);
                                       check the result with umgs_frame_check */
    UMGS_RENDER_DEPTH = 16,         /* FULL mode only, needs a frame: also keep each pixel's expected
                                       depth sum_i w_i z_i / sum_i w_i over its blended fragments (w_i
                                       the blend weight of Eq. 2 or Eq. 9, z_i the camera depth of a
                                       Gaussian's mean or a triangle's perspective-correct depth at the
                                       pixel centre; +inf where nothing blends), for umgs_frame_depth;
                                       not with SAVE_BACKWARD, MIXED or T_PRODUCT. */
    UMGS_RENDER_SOFT_EDGE = 32      /* FULL mode only (an extension beyond the paper): the binary sample
                                       coverage o^j of Eq. 7-8 becomes c^j = prod_e sigmoid(d_e / edge_sigma),
                                       d_e the signed distance in pixels (positive inside) from sample j to
                                       edge e of the unsnapped projected triangle; a triangle is a fragment
                                       of every pixel of its pixel rect widened by ceil(8 edge_sigma) pixels
                                       and Eq. 7-9 use c for o.  With SAVE_BACKWARD, umgs_render_backward
                                       also carries the gradient through c to the vertex positions.
                                       Needs 0 < edge_sigma <= 16; not with MIXED, T_PRODUCT, DEPTH or a
                                       persistent schedule (sched > 0).  Grid launch of its own compositor. */
};

typedef struct {
    int32_t tile_size;       /* 8, 16 or 32 pixels; 0 = 16 */
    int32_t blend_mode;      /* UMGS_BLEND_* */
    float t_eps;             /* early termination: stop after T < t_eps; 0 = never (default 1e-4) */
    float bg[3];             /* opaque background colour (Eq. 10-11) */
    int32_t flags;           /* UMGS_RENDER_* bits */
    int32_t sched;           /* compositor schedule: 0 = one CTA per tile; k > 0 = persistent launch with
                                k CTAs per SM taking tiles in decreasing order of list length */
    float edge_sigma;        /* UMGS_RENDER_SOFT_EDGE: edge width sigma in pixels (default 0) */
    int32_t split;           /* per-tile work split for uneven loads: 0 = off; else 256..1048576, a tile
                                whose list holds more than `split` records is composited as segments of
                                `split` records on separate CTAs, each from T = 1, merged per pixel front
                                to back (C = sum_k (prod_{m<k} T_m) C_k).  Cuts only in front of a list's
                                first triangle record (entity state of Eq. 7-9 never crosses a cut).  The
                                fp association differs from the whole tile, and a segment stops at its own
                                T < t_eps: pixels agree with the whole-tile composite within t_eps times the
                                largest colour plus rounding.  Not with SAVE_BACKWARD, DEPTH or SOFT_EDGE.
                                Up to 65,535 segments (512 MB of segment buffers) per render; tiles beyond
                                that are composited whole. */
} umgs_render_opts;

/* Gradient outputs of umgs_render_backward; every pointer is nullable (not
 * computed).  Shapes follow the inputs; all float32. */
typedef struct {
    float* means;      /* [n,3] */
    float* quats;      /* [n,4]  (when the render used quats/scales) */
    float* scales;     /* [n,3] */
    float* opacities;  /* [n] */
    float* sh;         /* [n,(deg+1)^2,3] */
    float* cov3d;      /* [n,6]  (when the render used cov3d) */
} umgs_gaussian_grads;

typedef struct {
    float* verts;      /* [nv,3] (through attribute interpolation; through the sample coverage too
                          after a UMGS_RENDER_SOFT_EDGE render, binary coverage being piecewise constant) */
    float* vcolor;     /* [nv,3] */
    float* valpha;     /* [nv]   (when the mesh has valpha and no falpha) */
    float* falpha;     /* [nf]   (when the mesh has falpha) */
} umgs_mesh_grads;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  Synchronises. */
umgs_status umgs_ctx_create(umgs_ctx** out, int device);
/* Destroy a context and free its workspace.  Synchronises the device. */
void umgs_ctx_destroy(umgs_ctx* ctx);
/* Last error message of this context ("" after success). */
const char* umgs_last_error(const umgs_ctx* ctx);
/* Synchronise `stream` and report any error a kernel of this context
 * detected on the device since the previous umgs_ctx_sync (deferred
 * argument errors of asynchronous calls such as umgs_deform). */
umgs_status umgs_ctx_sync(umgs_ctx* ctx, void* stream);
/* Default render options (tile 16, FULL, t_eps 1e-4, black background). */
void umgs_default_render_opts(umgs_render_opts* opts);

/* A frame holds the projected records, sorted tile lists and per-pixel state
 * of one umgs_render call, for umgs_render_backward and for inspection.  A
 * frame is used with its context only while that context lives; destroying
 * it (umgs_frame_destroy) is allowed after its context was destroyed. */
umgs_status umgs_frame_create(umgs_ctx* ctx, umgs_frame** out);
void umgs_frame_destroy(umgs_frame* frame);

/* ---- rendering (Sec. 3.2, Eq. 1-2 and 7-11) -------------------------------
 *
 * Renders ncams views of the Gaussians and nmeshes meshes in ONE pass per
 * view: Gaussians are EWA-projected to 2D conics, triangles are set up with
 * integer edge functions over 4 samples per pixel; every primitive is binned
 * into the lists of the screen tiles its footprint touches, each list in
 * (depth bits, unified id) order (records sorted by depth once, then binned
 * through regions of 8 x 4 tiles), and each pixel composites its
 * depth-ordered fragments front to back.  A run of
 * depth-adjacent triangle fragments with no Gaussian between them forms one
 * entity whose sub-pixel transmittances t^j give the continuous coverage
 * O_i (Eq. 7-9); T after an entity is T_in * mean_j t^j.  Gaussian alpha is
 * min(0.99, o*exp(-d^T conic d / 2)), fragments below 1/255 are skipped.
 *
 * gaussians  host pointer to a umgs_gaussians (n may be 0)
 * meshes     host array of nmeshes umgs_mesh (may be NULL when nmeshes == 0)
 * cams       host array of ncams cameras; all must have the same width/height
 * opts       host pointer; NULL = defaults
 * out_rgbt   [ncams,H,W,4] device float, 16-byte aligned: RGB (background
 *            included) and the final transmittance T
 * frame      nullable; when given, the frame keeps everything
 *            umgs_render_backward needs (and the call uses its buffers)
 * Synchronises once per call on `stream` to read the number of keys, except
 * with UMGS_RENDER_ASYNC (then asynchronous on `stream`; the frame must have
 * a pair capacity from umgs_frame_reserve, the number of keys is not known
 * on the host afterwards, and a render that needs more pairs composites no
 * tile and is reported by umgs_frame_check).
 * Errors: INVALID_ARG (NULL arrays with n > 0, misaligned out_rgbt or sh,
 * ncams < 1, mixed image sizes,
 * image sides above 32768, tile_size not 8/16/32, sh_degree > 3, more than
 * 4294967294 primitives, more than 2^22 regions of 8 x 4 tiles over the
 * cameras, ASYNC without a frame or capacity), CAPACITY (more than
 * 4294967294 (tile, primitive) list entries), OUT_OF_MEMORY, CUDA.
 */
umgs_status umgs_render(umgs_ctx* ctx, const umgs_gaussians* gaussians,
                        const umgs_mesh* meshes, int32_t nmeshes,
                        const umgs_camera* cams, int32_t ncams,
                        const umgs_render_opts* opts, float* out_rgbt,
                        umgs_frame* frame, void* stream);

/* Number of keys (tile, primitive) pairs and tiles (all cameras) of the last
 * render into `frame` (num_keys = -1 after an asynchronous render).  Host
 * outputs; synchronises nothing. */
umgs_status umgs_frame_counts(const umgs_frame* frame, int64_t* num_keys, int64_t* num_tiles);

/* Pair capacity of asynchronous renders (UMGS_RENDER_ASYNC) into `frame`:
 * the pair buffers are sized to key_capacity at the next such render (an
 * allocation at most once per growth).  A capacity from a synchronous
 * render's count with some headroom (e.g. 1.25 x) suits a scene whose
 * footprints change little between calls.  Errors: INVALID_ARG
 * (key_capacity < 1). */
umgs_status umgs_frame_reserve(umgs_frame* frame, int64_t key_capacity);

/* Expected depth of every pixel of the last render into `frame` made with
 * UMGS_RENDER_DEPTH (see the flag): out_depth [ncams,H,W] float device
 * (caller-owned); asynchronous on `stream`.  Errors: INVALID_ARG (no such
 * render), CUDA. */
umgs_status umgs_frame_depth(const umgs_frame* frame, float* out_depth, void* stream);

/* Separate-pass baseline (the scheme Sec. 4.1 and Fig. 5b compare against;
 * not a step of the method): two layers rendered apart, each with a zero
 * background and UMGS_RENDER_DEPTH, composited per pixel in the order of
 * their expected depths (the nearer layer over the farther, layer a first
 * on equal depths), then the background bg:
 *   C = C_f + T_f C_b + T_f T_b bg,  T = T_f T_b.
 * a_rgbt, b_rgbt, out_rgbt [npix,4] (16-byte aligned) and a_depth, b_depth [npix] float device;
 * bg host float[3].  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
umgs_status umgs_composite_layers(umgs_ctx* ctx, const float* a_rgbt, const float* a_depth, const float* b_rgbt,
                                  const float* b_depth, int64_t npix, const float* bg, float* out_rgbt,
                                  void* stream);

/* Synchronises `stream` and reports the device-side conditions of the last
 * render into `frame`: CAPACITY if it needed more pairs than the reserved
 * capacity (that render composited no tile: background, T = 1; reserve more
 * and render again), INVALID_ARG for an out-of-range face index, TIMEOUT if
 * a wait of the binning stage's single-sweep kernels (a block waiting for
 * the prefix published by the blocks before it, bounded to about 2^20 polls)
 * gave up; its lists are then not valid. */
umgs_status umgs_frame_check(umgs_frame* frame, void* stream);

/* Number of (pixel, fragment) evaluations of the last render into `frame`:
 * for every pixel, the entries of its tile list whose footprint (Gaussian
 * pixel rect, triangle pixel rect) holds the pixel, up to and including the
 * one after which T < t_eps.  The algorithmic work unit of the compositor
 * (N_alg).  Counted by one diagnostic kernel over the saved tile lists (the
 * render itself counts nothing); host output; synchronises `stream`. */
umgs_status umgs_frame_evaluations(const umgs_frame* frame, int64_t* evals, void* stream);

/* Counters of the last render into `frame` (diagnostic; host output;
 * synchronises `stream`):
 *   gaussian_evals, triangle_evals: umgs_frame_evaluations split by the kind
 *     of record (their sum is N_alg); the compositor's work differs per kind
 *     (a Gaussian evaluation is an exponential and a blend, Eq. 1-2; a
 *     triangle evaluation is 12 sample/edge tests, perspective-correct
 *     attributes and the entity blend, Eq. 7-9);
 *   fp64_conics: (camera, Gaussian) records whose projected covariance was
 *     near-singular (det < a c / 128) and whose conic was therefore inverted
 *     in fp64 (EWA projection, Sec. 3.2);
 *   list_entries: total length of the tile lists.
 * Errors: INVALID_ARG if nothing was rendered into the frame. */
typedef struct {
    int64_t gaussian_evals;
    int64_t triangle_evals;
    int64_t fp64_conics;
    int64_t list_entries;
} umgs_frame_stats;
umgs_status umgs_frame_stats_read(const umgs_frame* frame, umgs_frame_stats* out, void* stream);

/* Copy the sorted tile lists of the last render into caller buffers (device):
 * tile_ptr [num_tiles+1] int64 (list of tile t is [tile_ptr[t], tile_ptr[t+1])),
 * ids [num_keys] int32 unified primitive ids, dbits [num_keys] uint32 depth
 * bits; each list in ascending (depth bits, id).  Asynchronous on stream. */
umgs_status umgs_frame_lists(const umgs_frame* frame, int64_t* tile_ptr, int32_t* ids,
                             uint32_t* dbits, void* stream);

/* ---- backward (gradient of the composite) ----------------------------------
 *
 * Given dL/d(out_rgbt) of a umgs_render call that used a frame and the flag
 * UMGS_RENDER_SAVE_BACKWARD (blend mode FULL), computes dL/d of the inputs:
 * Gaussian means, quats, scales (or cov3d), opacities, SH; mesh vertex
 * positions (through the perspective-correct attribute interpolation), vertex
 * colours and alphas (vertex positions also through the sample coverage
 * after a UMGS_RENDER_SOFT_EDGE render).  The sorted lists of the frame are replayed back to
 * front per pixel; Gaussian transmittance is recovered by division
 * (alpha <= 0.99), triangle entities use the per-pixel stack of sub-sample
 * transmittances saved by the forward, so opaque triangles need no division.
 * The derivative is that of the function the forward computed (early
 * termination included); clamps (alpha max 0.99, alpha to [0,1], colour >= 0,
 * barycentrics >= 0) pass the gradient at their boundary.
 *
 * frame      the frame of the forward call (same ctx)
 * g, meshes  the SAME inputs as the forward call
 * dL_drgbt   [ncams,H,W,4] device float, 16-byte aligned: dL/dR, dL/dG, dL/dB, dL/dT
 *            (g->quats, when used, and gg->quats are read and written as
 *            16-byte rows: both 16-byte aligned)
 * gg, mg     host structs of device output pointers (mg: nmeshes entries);
 *            outputs are overwritten (zero-filled first)
 * Synchronises once (checks the saved-state capacity; if a pixel had more
 * triangle fragments than the stack held, the forward composite is re-run
 * with a larger stack first).  Errors: INVALID_ARG (no saved frame, sizes, alignment),
 * NOT_IMPLEMENTED (blend modes other than FULL), OUT_OF_MEMORY, CUDA.
 */
umgs_status umgs_render_backward(umgs_ctx* ctx, umgs_frame* frame, const umgs_gaussians* g,
                                 const umgs_mesh* meshes, int32_t nmeshes, const float* dL_drgbt,
                                 const umgs_gaussian_grads* gg, const umgs_mesh_grads* mg, void* stream);

/* ---- Gaussian-centric binding (Sec. 3.3, "Binding Gaussians to Mesh") -------
 *
 * For every Gaussian, one target (mode CENTER: the mean; the paper's
 * UniMGS*) or 8 targets (mode BBX: the corners mu + R_q (+-k s_x, +-k s_y,
 * +-k s_z), corner c taking the + sign on axis j when bit j of c is set; the
 * paper's UniMGS).  From every camera centre o a ray o + t (p - o), t > 0, is
 * cast through the target p; every proxy face it hits is a candidate and the
 * target binds to the hit nearest to p (distance |t - 1| |p - o|; ties:
 * lower camera index, then lower face index).  A target that no ray hits,
 * and every target in mode NEAREST, binds to the closest point of the proxy
 * mesh (ties: lower face index).  The ray/triangle test (Moller-Trumbore)
 * and the closest-point evaluation use canonical float32 operations, so the
 * result equals a brute-force search over all faces and cameras bit for bit.
 *
 * g          Gaussians (means; quats and scales in mode BBX)
 * proxy_v    [nv,3], proxy_f [nf,3] int32
 * cams       host array of ncams cameras (only the pose is used; ignored in NEAREST)
 * k_sigma    box half-size in standard deviations (the paper's BBX; 3)
 * out_face   [n,8] int32 bound face per target (CENTER/NEAREST: 8 copies)
 * out_bary   [n,8,2] (b1, b2): the bound point is (1-b1-b2) v0 + b1 v1 + b2 v2
 * out_dist   [n,8] distance from the target to the bound point
 * out_flags  [n,8] uint8: 1 = ray hit, 2 = closest-point fallback / NEAREST
 * out_num_fallback  host; number of [n,8] slots with flag 2 (nullable)
 * Synchronises (reads the grid size and the fallback count).  Errors:
 * INVALID_ARG (sizes, NULL arrays, out-of-range proxy face ids), CAPACITY
 * (a ray exceeded the cell-visit budget), OUT_OF_MEMORY, CUDA.
 */
umgs_status umgs_bind(umgs_ctx* ctx, const umgs_gaussians* g, const float* proxy_v, const int32_t* proxy_f,
                      int64_t nv, int64_t nf, const umgs_camera* cams, int32_t ncams, int32_t mode, float k_sigma,
                      int32_t* out_face, float* out_bary, float* out_dist, uint8_t* out_flags,
                      int64_t* out_num_fallback, void* stream);

/* ---- deformation transfer (Sec. 3.3, Eq. 12-13) ---------------------------
 *
 * Per proxy face f: deformation gradient D_f = F'_f F_f^-1 with the frame
 * F = [e1, e2, n/sqrt(|n|)] (e1 = v1-v0, e2 = v2-v0, n = e1 x e2; the frames
 * and the inverse are computed in fp64 for sliver faces).  Per proxy vertex: D_v = rest-area-
 * weighted mean of the incident D_f, polar D_v = R_v S_v (a proper rotation;
 * for det D_v < 0 the smallest singular direction is flipped), r_v = log R_v
 * (axis-angle, angle in [0, pi]), Delta_v = V'_v - V_v.
 * Per Gaussian, for each of its 8 bound points P_i (face[i], barycentrics
 * (1-b1-b2, b1, b2) on the face's vertices 0,1,2): Delta_i, r_i, S_i by
 * barycentric interpolation (Eq. 12); R' = exp(mean r_i), S' = mean S_i
 * (Eq. 13); Sigma' = (R'S') Sigma (R'S')^T; q' = quat(R') * q (w >= 0);
 * mu' = mu + mean Delta_i (mode LITERAL, Eq. 13 as printed) or
 * mu' = mu + mean Delta_i + (R'S' - I)(mu - mean P_i) (mode FRAME, default:
 * exact for rigid motions and uniform scalings of the proxy).
 * With UMGS_DEFORM_ONE_RING in `mode` (closer to ACAP's own per-vertex fit)
 * D_v is instead the cotangent-weighted least-squares map of the vertex's
 * one-ring edges plus its normal:
 *   D_v = (sum_j c_vj e'_vj e_vj^T + n'_v n_v^T)(sum_j c_vj e_vj e_vj^T + n_v n_v^T)^-1
 * (e_vj = V_j - V_v, c_vj = sum over the edge's faces of max(0, cot/2) of the
 * opposite angle, N_v = sum of e1 x e2 over the faces at v, n_v = N_v/sqrt|N_v|;
 * primes: deformed); the rest is unchanged.
 *
 * rest       Gaussians at rest (means, quats, scales or cov3d; n); SH/opacity unused
 * face       [n,8] int32 proxy face per bound point (from umgs_bind)
 * bary       [n,8,2] float (b1, b2) per bound point (from umgs_bind)
 * proxy_v    [nv,3] rest proxy vertices; proxy_vd [nv,3] deformed vertices
 * proxy_f    [nf,3] int32 proxy faces
 * out_means  [n,3]; out_cov3d [n,6] (xx,xy,xz,yy,yz,zz); out_quats [n,4] (nullable)
 * Asynchronous.  Errors: INVALID_ARG (NULL arrays, nv < 3 or nf < 1, bad
 * mode), OUT_OF_MEMORY, CUDA.  A face id outside [0,nf) or a proxy vertex
 * index outside [0,nv) is detected on the device: the affected outputs are
 * NaN and the next umgs_ctx_sync reports INVALID_ARG.
 */
umgs_status umgs_deform(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* face, const float* bary,
                        const float* proxy_v, const float* proxy_vd, const int32_t* proxy_f, int64_t nv,
                        int64_t nf, int32_t mode, float* out_means, float* out_cov3d, float* out_quats,
                        void* stream);

/* The per-vertex transform table of the last umgs_deform call, copied to a
 * caller buffer [nv,12] (Delta xyz, r xyz, S xx xy xz yy yz zz).  Async. */
umgs_status umgs_deform_vertex_table(umgs_ctx* ctx, float* out_table, int64_t nv, void* stream);

/* Number of proxy faces of the last umgs_deform / umgs_deform_compact on
 * `ctx` whose rest frame [e1, e2, n/sqrt|n|] was a sliver (|e1 x e2| <
 * 1e-3 |e1||e2|), whose deformation gradient (both frames and the inverse)
 * was therefore computed in fp64 (per-face deformation
 * gradient of the per-vertex transform, Sec. 3.3).  Host output;
 * synchronises `stream`. */
umgs_status umgs_deform_fp64_faces(umgs_ctx* ctx, int64_t* count, void* stream);

/* Compact binding: a regrouping of Eq. 12-13, not a step of the paper.
 * Every interpolant that Eq. 13 averages is linear in the proxy vertex
 * rows, so a Gaussian's deformation needs only its distinct bound vertices v
 * and the weights w_v = (1/8) x (sum over its 8 bound points of the
 * barycentric weight of v).  umgs_binding_compact derives them once from a
 * binding as umgs_bind writes it (face [n,8], bary [n,8,2]) and the proxy
 * faces:
 *   out_count   [n] int32 device: distinct vertices (1..24), or -1 for an
 *               out-of-range face or vertex index
 *   out_entries [n,24,2] int32 device: (vertex id, weight as float bits);
 *               the first out_count[i] are used, in order of first appearance
 * umgs_deform_compact is umgs_deform (same modes, outputs and errors; NaN and
 * a status bit for a -1 count) over that form: about 10 vertex rows gathered
 * per Gaussian instead of 24; it agrees with umgs_deform up to fp32
 * summation order.  Both asynchronous on `stream`; bary 8-byte aligned, the
 * entries 8-byte aligned for umgs_binding_compact and 16-byte aligned for
 * umgs_deform_compact (it reads two entries per load).  Errors: INVALID_ARG
 * (sizes, NULL arrays, alignment), CUDA. */
umgs_status umgs_binding_compact(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n,
                                 const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t* out_count,
                                 int32_t* out_entries, void* stream);
umgs_status umgs_deform_compact(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* count,
                                const int32_t* entries, const float* proxy_v, const float* proxy_vd,
                                const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t mode, float* out_means,
                                float* out_cov3d, float* out_quats, void* stream);

/* The compact binding packed without padding (CSR): Gaussian i's distinct
 * vertices and weights are entries [offsets[i], offsets[i+1]) of one array,
 * in order of first appearance, each run padded to an even length with a
 * zero-weight copy of its first entry (about 11 entries per Gaussian for the
 * 1080p workload instead of 24 padded rows: the deformation reads 88 bytes
 * per Gaussian, not 192-byte rows).  A Gaussian with an out-of-range face or
 * vertex index gets the entries (-1, 0), (-1, 0).
 *   out_offsets [n+1] int32 device; out_entries [cap,2] int32 device
 *   (vertex id, weight as float bits), 16-byte aligned, nullable if cap = 0;
 *   *out_total (host): the entries needed.
 * Synchronises `stream`.  Errors: INVALID_ARG, CAPACITY when *out_total >
 * cap (offsets written, entries not: call again with a larger buffer), CUDA.
 * umgs_deform_csr is umgs_deform_compact over that form (same modes, outputs
 * and errors). */
umgs_status umgs_binding_csr(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n,
                             const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t* out_offsets,
                             int32_t* out_entries, int64_t cap, int64_t* out_total, void* stream);
umgs_status umgs_deform_csr(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* offsets,
                            const int32_t* entries, const float* proxy_v, const float* proxy_vd,
                            const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t mode, float* out_means,
                            float* out_cov3d, float* out_quats, void* stream);

/* Spatial order of n Gaussians (a layout tool; no paper counterpart):
 * out_perm[i] = the index of the Gaussian that comes i-th in the order of the
 * 30-bit Morton code of its mean (10 bits per axis over the bounding box of
 * the finite means: q = trunc(clamp((x - lo) * (1024 / (hi - lo)), 0, 1023)),
 * a non-finite coordinate counts as lo; equal codes in index order).  A
 * model stored in that order (every per-Gaussian array gathered by out_perm
 * once, when it is loaded, before the binding) keeps Gaussians that are close
 * in space close in memory: the deformation's gathers of proxy-vertex rows
 * then hit the cache.  The renderer's results do not depend on the order
 * beyond the unified ids that break exact depth ties.
 *   means [n,3] float device; out_perm [n] int32 device.
 * Synchronises `stream`; keeps a workspace of 16 n bytes in the context and
 * sorts with the sort workspace of the context's default frame (the one
 * umgs_render uses when given no frame), so it must not run while a render
 * into that frame is in flight on another stream.
 * Errors: INVALID_ARG (NULL arrays, n < 0 or n >= 2^31 - 1), OUT_OF_MEMORY,
 * CUDA. */
umgs_status umgs_spatial_order(umgs_ctx* ctx, const float* means, int64_t n, int32_t* out_perm, void* stream);

/* ---- multi-view form: CUDA graph and autotuning -----------------------------
 *
 * umgs_render_graph_create renders once (an ordinary umgs_render into
 * `frame`, which sizes every buffer and uploads the cameras), then captures
 * the same render into a CUDA graph on a private stream.  The captured render
 * has no host read-back: the (tile, primitive) pair buffers hold
 * key_headroom (>= 1; default 1.25) times the pairs of the sizing render,
 * and a larger count is flagged on the device instead of being written.
 * umgs_graph_launch replays it asynchronously on `stream` with the SAME
 * input and output device pointers and the cameras of the creation call
 * (their contents may change between launches, the cameras may not);
 * umgs_graph_check synchronises `stream` and reports CAPACITY if a launch
 * needed more pairs (re-create the graph; that launch composited no tile, so
 * its output is the background with T = 1), INVALID_ARG for bad face indices.
 * The frame belongs to the graph until umgs_graph_destroy.
 */
typedef struct umgs_graph umgs_graph;
umgs_status umgs_render_graph_create(umgs_ctx* ctx, umgs_frame* frame, const umgs_gaussians* gaussians,
                                     const umgs_mesh* meshes, int32_t nmeshes, const umgs_camera* cams,
                                     int32_t ncams, const umgs_render_opts* opts, float* out_rgbt,
                                     float key_headroom, umgs_graph** out, void* stream);
umgs_status umgs_graph_launch(umgs_graph* graph, void* stream);
umgs_status umgs_graph_check(umgs_graph* graph, void* stream);
void umgs_graph_destroy(umgs_graph* graph);

/* Autotuner: renders the given workload with every tile size (8, 16, 32),
 * compositor schedule (one CTA per tile; persistent with 1, 2 or 4 CTAs
 * per SM; one CTA per tile only with UMGS_RENDER_SOFT_EDGE) and per-tile
 * work split (off, 512, 1024, 2048 records; off with SOFT_EDGE, DEPTH or
 * SAVE_BACKWARD), 1 warm-up + 3 timed renders each (CUDA events on
 * `stream`), and writes the fastest tile_size, sched and split into *inout
 * (other fields kept) and
 * its time in ms per render into *best_ms (nullable).  out_rgbt receives the
 * renders ([ncams,H,W,4]).  Synchronises. */
umgs_status umgs_autotune(umgs_ctx* ctx, const umgs_gaussians* gaussians, const umgs_mesh* meshes,
                          int32_t nmeshes, const umgs_camera* cams, int32_t ncams, umgs_render_opts* inout,
                          float* out_rgbt, double* best_ms, void* stream);

/* ---- per-stage timing ------------------------------------------------------
 * When enabled, every stage launched by this context is bracketed by CUDA
 * events recorded on the stream it runs on.  umgs_profile_read synchronises
 * those events, returns per stage the summed milliseconds and the number of
 * launches since the last read (host arrays of UMGS_NUM_STAGES), and clears
 * the record.  Stages: */
enum {
    UMGS_STAGE_PROJECT_GAUSSIANS = 0, UMGS_STAGE_SETUP_TRIANGLES, UMGS_STAGE_SCAN, UMGS_STAGE_SCATTER,
    UMGS_STAGE_SORT, UMGS_STAGE_COMPOSITE, UMGS_STAGE_DEFORM_FACES, UMGS_STAGE_DEFORM_VERTICES,
    UMGS_STAGE_DEFORM_GAUSSIANS, UMGS_STAGE_BIND_GRID, UMGS_STAGE_BIND_RAYCAST, UMGS_STAGE_BIND_NEAREST,
    UMGS_STAGE_BACKWARD_COMPOSITE, UMGS_STAGE_BACKWARD_PROJECT, UMGS_STAGE_SHADE_GAUSSIANS,
    UMGS_NUM_STAGES = 16
};
umgs_status umgs_profile_enable(umgs_ctx* ctx, int32_t on);
umgs_status umgs_profile_read(umgs_ctx* ctx, double* ms, int64_t* launches);

/* Number of kernels this library has launched in this process since it was
 * loaded, over all contexts and devices (a launch of a render graph adds the
 * number of kernels captured into it; capturing adds nothing).  Never fails;
 * thread-safe.  The difference of two reads counts the kernels launched in
 * between by the calling thread when no other thread uses the library. */
long long umgs_kernel_launches(void);

/* ---- deformation without device allocation ---------------------------------
 * No counterpart in the paper.  For callers that cannot allocate device
 * memory - e.g. a host application that hands all device memory to its own
 * allocator at start-up, a plugin in a process whose device memory another
 * runtime owns, or a real-time loop that cannot absorb the synchronisation
 * of cudaMalloc - this computes exactly what umgs_deform computes (same
 * kernels, same arguments, same output layout) without a context and
 * without calling cudaMalloc, cudaFree or any allocating routine.
 *
 * Its scratch (per-vertex accumulators, the vertex transform table and a
 * status word) lives in one file-scope __device__ array sized for
 * UMGS_NOALLOC_MAX_PROXY_VERTICES proxy vertices (about 3.4 MB), which every
 * GPU that loads the library keeps until the process exits.
 *  - Runs on the CALLING thread's current device and on `stream`.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: after cudaDeviceReset (or any other teardown of the device's
 *    primary context) the array may move and this entry point must not be
 *    called again on that device in this process.
 *  - All calls share the array and it keeps the last call's contents (each
 *    call clears what must start at zero): calls that overlap on the GPU
 *    (several streams or host threads at once) race and give wrong results.
 *  - Out-of-range face or vertex ids give NaN outputs for the affected
 *    Gaussians; no deferred status is kept.
 *  - The per-face transform only: UMGS_DEFORM_ONE_RING is rejected.
 * Errors: INVALID_ARG (as umgs_deform, and ONE_RING), CAPACITY (nv above the
 * maximum), CUDA (lookup or launch failure).  Asynchronous.
 */
#define UMGS_NOALLOC_MAX_PROXY_VERTICES 32768
umgs_status umgs_deform_noalloc(const umgs_gaussians* rest, const int32_t* face, const float* bary,
                                const float* proxy_v, const float* proxy_vd, const int32_t* proxy_f,
                                int64_t nv, int64_t nf, int32_t mode, float* out_means, float* out_cov3d,
                                float* out_quats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UMGS_H */
