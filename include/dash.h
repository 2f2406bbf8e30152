/*
 * dash.h — C ABI of the GB300 (sm_103a) Dash streaming PARAFAC2 library.
 *
 * Dash (Jang, Jang and Kang, KDD'23) keeps a PARAFAC2 model X_k ≈ U_k S_k Vᵀ
 * of an irregular tensor {X_k} up to date while new rows of existing slices
 * and whole new slices arrive (§2.2, Problem 1).  Each call to dash_update()
 * is one "update" of Figure 3: it absorbs every row staged since the previous
 * update with one pass of Algorithm 1, touching only the new rows and the
 * λ-weighted helper summaries c_k, D_k, F, G (§3.2, Eqs. 11-21).
 *
 * Two model forms share the interface:
 *   DASH_MODE_P  Algorithm 1 as written (U_k free).
 *   DASH_MODE_Q  the constrained form U_k = Q_k H S_k with column-orthonormal
 *                Q_k (the reparameterisation mentioned in §2.1), streamed
 *                with the same old/new split (see dash_update()).
 *
 * Conventions for every entry point
 *   - All matrices are row-major, dense, 0-based.  V is J×R, W is K×R
 *     (row k = diagonal of S_k), D_k is R×R, F is J×R, G and H are R×R,
 *     Z_k is R×J.  Row block X_k,new is I_k,new×J with leading dimension ld
 *     (elements, >= J).
 *   - Host pointers are read or written before the call returns; device
 *     pointers (`where == DASH_DEVICE`) are read in stream order on the
 *     model's stream.  The library never frees caller memory.
 *   - Every call returns a dash_status.  On an error the model keeps its
 *     previous state (argument and capacity errors are found on the host
 *     before any device work) and dash_last_error() describes the cause.
 *     A CUDA error (DASH_ECUDA) leaves the model unusable: destroy it.
 *   - A model is not thread-safe; calls on one model must be serialised.
 */
#ifndef DASH_H
#define DASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dash_model dash_model;

typedef enum dash_status {
    DASH_OK = 0,
    DASH_EINVAL = 1,     /* bad argument (shape, id, dtype, null pointer)   */
    DASH_ENOMEM = 2,     /* device allocation failed or a capacity exceeded */
    DASH_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed      */
    DASH_ESTATE = 4,     /* call not valid now (e.g. V never set)            */
    DASH_ENUMERIC = 5,   /* a non-finite value reached the factors (reported
                            by the next fitness/state read or update)        */
    DASH_ETIMEOUT = 6    /* a bounded device wait gave up                    */
} dash_status;

enum { DASH_MODE_P = 0, DASH_MODE_Q = 1 };

/* Arithmetic of the bulk products X_new·V and X_newᵀ(U S) (Theorem 1's
 * dominant terms).  R×R solves, summaries and fitness are FP64 in all three. */
enum {
    DASH_PREC_FP64 = 0,  /* FP64 products                                      */
    DASH_PREC_FP32 = 1,  /* FP32 products, FP32 accumulation                   */
    DASH_PREC_F16X3 = 2  /* tensor cores: FP16 hi/lo split, 3 products, FP32 acc  */
};

enum { DASH_F64 = 0, DASH_F32 = 1 };        /* element type of staged X   */
enum { DASH_HOST = 0, DASH_DEVICE = 1 };    /* where a caller pointer lives */

typedef struct dash_config {
    int32_t J;              /* columns of every slice (> 0)                      */
    int32_t R;              /* target rank, 1..64                                */
    double lambda;          /* forgetting factor λ, 0 < λ <= 1 (Eq. 5)           */
    int32_t mode;           /* DASH_MODE_P or DASH_MODE_Q                        */
    int32_t precision;      /* DASH_PREC_*                                       */
    int32_t input_dtype;    /* DASH_F64 or DASH_F32: element type of X           */
    int32_t n_sweeps;       /* passes of Algorithm 1 per update, 1..64 (mode P;
                               mode Q runs one)                                */
    double pinv_rtol;       /* pseudo-inverse cut-off relative to the largest
                               singular value; <= 0 selects R·DBL_EPSILON      */
    int64_t max_slices;     /* capacity K_max of slices over the model's life    */
    int64_t max_rows;       /* capacity of rows per update (scratch sizing)      */
    int64_t max_segments;   /* capacity of segments per update                   */
    void *stream;           /* cudaStream_t to run on; NULL = a private stream   */
    int64_t max_staged_rows;/* rows each of the two append_* staging buffers
                               holds; 0 = max_rows (device-resident batches
                               need no staging)                                */
} dash_config;

/* Fill *cfg with defaults for (J, R, λ): mode P, FP32 products, FP32 input,
 * one sweep, capacities 1<<16 slices / 1<<20 rows / 1<<17 segments. */
void dash_config_default(dash_config *cfg, int32_t J, int32_t R, double lambda);

/* init(K, J, R, λ) of the problem statement: create a model with no slices.
 * Allocates all device memory for the capacities in cfg (DASH_ENOMEM if it
 * does not fit).  V must be set with dash_set_factors() or dash_set_state()
 * before the first update. */
dash_status dash_init(const dash_config *cfg, dash_model **out);
void dash_destroy(dash_model *m);
const char *dash_last_error(const dash_model *m);
const char *dash_status_string(dash_status s);

/* Set the shared factors from host FP64 arrays: V (J×R) and, in mode Q,
 * H (R×R; NULL = identity).  Used for a fresh model (the starting V of the
 * static fit, §3.2.1). */
dash_status dash_set_factors(dash_model *m, const double *V, const double *H);

/* Replace the whole mode-P state (host FP64): K slices with factors V, W and
 * helpers c (K×R), D (K×R×R), F (J×R), G (R×R) of §3.2.1 (Eqs. 6-9).  This
 * is how a model resumes from saved or externally initialised helpers. */
dash_status dash_set_state_p(dash_model *m, int64_t K, const double *V, const double *W,
                             const double *c, const double *D, const double *F,
                             const double *G);
/* Read the mode-P state into host FP64 arrays sized for the current K
 * (dash_num_slices()).  Any pointer may be NULL to skip that array. */
dash_status dash_get_state_p(const dash_model *m, double *V, double *W, double *c,
                             double *D, double *F, double *G);

/* Mode-Q state (host FP64): V (J×R), H (R×R), W (K×R) and, per slice,
 *   L_k (K×R×R): upper-triangular with a non-negative diagonal, the R factor
 *     of the λ^{age/2}-weighted stacked A rows, so L_kᵀL_k = B_k =
 *     Σ λ^age A_kᵀA_k;
 *   Y_k (K×R×J): the projected data Y_k = T_k Z_k = Q_kᵀΛ_kX_k with
 *     T_k = B_k^{-1/2} and Z_k = Σ λ^age A_kᵀX_k.
 * Neither B_k nor Z_k is held: B_k has condition number cond(A_k)², which on
 * U(0,1) planted factors reaches 1e9-1e12, and T_k·Z_k formed in low
 * precision cancels catastrophically; L_k and Y_k are well scaled.
 * set_state_q rejects an L_k with non-zero entries below the diagonal
 * (DASH_EINVAL) and derives each slice's eigenbasis from L_k.  Mode P models
 * return DASH_ESTATE.  get_state_q pointers may be NULL to skip an array. */
dash_status dash_set_state_q(dash_model *m, int64_t K, const double *V, const double *H,
                             const double *W, const double *L, const double *Y);
dash_status dash_get_state_q(const dash_model *m, double *V, double *H, double *W,
                             double *L, double *Y);

int64_t dash_num_slices(const dash_model *m);

/* append_rows(k, X_k,new): stage I_new new rows of existing slice k (or of a
 * slice staged by dash_append_slices() in this update).  Rows are appended
 * after the slice's existing rows, in call order.  X has input_dtype
 * elements, I_new×J with leading dimension ld, at `where`; it is copied. */
dash_status dash_append_rows(dash_model *m, int64_t k, const void *X, int64_t I_new,
                             int64_t ld, int32_t where);

/* append_slices({X_k}): stage L new slices with I[l] rows each (0 allowed);
 * they get ids K..K+L-1 (K = slices before this call plus earlier staged
 * new slices), returned in *first_new_id.  X[l] has leading dimension ld[l]
 * (NULL = J for all). */
dash_status dash_append_slices(dash_model *m, int64_t L, const int64_t *I,
                               const void *const *X, const int64_t *ld, int32_t where,
                               int64_t *first_new_id);

/* Stage a whole batch in CSR form in one call: segment s covers rows
 * row_ptr[s]..row_ptr[s+1]-1 of X (row-major, ld = J) and belongs to slice
 * slice_ids[s]; ids >= the current slice count (plus staged new slices)
 * create new slices, which must be numbered consecutively and appear in
 * ascending order.  slice_ids and row_ptr are host arrays; X is at `where`
 * and is copied (host → device with cudaMemcpyAsync; pinned memory lets
 * it overlap).  Staging alternates between two device buffers, so a batch
 * may be appended while the previous update still runs; a host X of 64 MiB
 * or more is split over several copy streams and copied in the background:
 * keep it unchanged until the next dash_update() returns. */
dash_status dash_append_batch(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                              const int64_t *row_ptr, const void *X, int32_t where);

/* One update of Algorithm 1 (mode P) or of the constrained stream (mode Q)
 * over everything staged since the last update, then clear the staging.
 * Mode P, in the order of Algorithm 1:
 *   U_k,new = X_k,new V S_k (S_k VᵀV S_k)⁺                 (Lemma 1, Eq. 11)
 *   c_k ← λc_k + vec(X_k,new)ᵀ(V ⊙ U_k,new),  D_k ← λD_k + U_k,newᵀU_k,new
 *   W(k,:) = c_kᵀ (VᵀV ∗ D_k)⁺  for every slice k        (Eqs. 15, 16, 12)
 *   F ← λF + Σ X_k,newᵀU_k,newS_k,  G ← λG + Σ S_kU_k,newᵀU_k,newS_k
 *   V = F G⁺                                              (Eqs. 20, 21, 17)
 * A new slice uses S_k = I in Lemma 1.  ⁺ is the Moore-Penrose
 * pseudo-inverse with cut-off pinv_rtol.
 * Mode Q: A_new = X_new V S_k Hᵀ; B_k ← λB_k + A_newᵀA_new (as
 *   L_k ← R factor of [√λ L_k; A_new]); Z_k ← λZ_k + A_newᵀX_new;
 *   T_k = B_k^{-1/2} (pseudo-inverse sense, from L_k); Q_k,new = A_new T_k;
 *   Y_k = T_k Z_k (carried as Y_k ← λ T_k,new B_k,old^{1/2} Y_k + Q_k,newᵀX_new);
 *   one CP-ALS sweep H → V → W on {Y_k}:
 *     H = (Σ Y_k V S_k)(VᵀV ∗ WᵀW)⁺,  V = (Σ Y_kᵀ H S_k)(HᵀH ∗ WᵀW)⁺,
 *     W(k,:) = diag(Hᵀ Y_k V)ᵀ (HᵀH ∗ VᵀV)⁺.
 *   The paper's Dash is unconstrained (§2.1 drops the Q_k H form); mode Q
 *   applies its old/new split to the constrained model.
 * Runs asynchronously on the model's stream; results are read by the
 * getters below, which synchronise. */
dash_status dash_update(dash_model *m);

/* The same update on a batch that already lives in device memory, read in
 * place (no staging copy): slice_ids/row_ptr as in dash_append_batch (host
 * arrays), X a device pointer of input_dtype, row-major with ld = J.  X must
 * stay unchanged until the update has run on the model's stream.  Nothing
 * may be staged when this is called. */
dash_status dash_update_device(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                               const int64_t *row_ptr, const void *X);

/* Static fit of the initial tensor (§3.2.1): on an empty model with the
 * staged batch made only of new slices, run n_iter ALS iterations from the
 * current V (each = one update on empty helpers, which equals one static
 * ALS iteration), then set the helpers from the final factors (Eqs. 6-9).
 * Clears the staging. */
dash_status dash_fit_initial(dash_model *m, int32_t n_iter);

/* dash_fit_initial() on a batch of new slices that lives in device memory,
 * read in place (same contract as dash_update_device()). */
dash_status dash_fit_initial_device(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                                    const int64_t *row_ptr, const void *X, int32_t n_iter);

/* factors(): copy V (J×R), rows k_first..k_first+k_count-1 of W, and in mode
 * Q H (R×R), to host FP64 arrays (NULL skips). */
dash_status dash_factors(const dash_model *m, double *V, double *W, int64_t k_first,
                         int64_t k_count, double *H);

/* New factor rows of the last update, in staging row order: U_k,new (mode P)
 * or Q_k,new (mode Q), N×R, to a host FP64 array.  *n_rows receives N. */
dash_status dash_new_rows(const dash_model *m, double *out, int64_t *n_rows);

/* fitness(): of the last update's batch with the updated factors,
 * fit = 1 − ||X_new − X̂_new||_F / ||X_new||_F with X̂_new = U_new S_k Vᵀ
 * (mode P, from FP64 Gram terms) or Q_new H S_k Vᵀ (mode Q, from a direct
 * residual pass accumulated in FP64).  x_norm2 (may be NULL) receives
 * ||X_new||²_F. */
dash_status dash_fitness(const dash_model *m, double *fit_batch, double *x_norm2);

/* λ-weighted fitness of every row absorbed so far (mode P), in the form that
 * Lemma 3's V step minimises (Eqs. 17, 20-21): each row x keeps the product
 * u·S_k that its own update produced (U_k,new S_k,new, frozen like the rows
 * of F and G) and is weighted by λ^age, age = updates since it arrived:
 *   fit_λ = 1 − sqrt(Σ λ^age ||x − (u∘w)Vᵀ||² / Σ λ^age ||x||²)
 * with the current V, evaluated from the helpers alone as
 *   Σ λ^age ||x − (u∘w)Vᵀ||² = xx − 2 tr(VᵀF) + tr(VᵀV G),  xx = Σ λ^age ||x||².
 * xx is tracked from every update's ||X_new||² (xx ← λ·xx + ||X_new||²),
 * starting at ||X_0||² after dash_fit_initial(); after dash_set_state_p() it
 * is unknown until dash_set_weighted_norm() supplies it (DASH_ESTATE until
 * then).  x_norm2_lambda (may be NULL) receives xx.  Mode Q: DASH_ESTATE.
 * Synchronises the stream. */
dash_status dash_fitness_lambda(const dash_model *m, double *fit_lambda, double *x_norm2_lambda);
/* Set xx = Σ λ^age ||x||² of the rows a loaded state summarises (part of the
 * resumable state together with dash_set_state_p()).  DASH_EINVAL if it is
 * negative or not finite. */
dash_status dash_set_weighted_norm(dash_model *m, double x_norm2_lambda);

/* Save the model's resumable state to a file: the configuration it was
 * created with (capacities included, the stream excluded), the slice count,
 * and the helpers an update reads as "old" (§3.2.1): mode P V, W, c_k, D_k,
 * F, G and xx; mode Q V, H, W, L_k, Y_k and each slice's eigenbasis and
 * B_k^{1/2} (so that the next update continues bit for bit), all as FP64,
 * followed by a checksum.  Nothing may be staged (DASH_ESTATE).  DASH_EINVAL
 * if the file cannot be written.  Synchronises the stream. */
dash_status dash_save(const dash_model *m, const char *path);
/* Create a model from a file written by dash_save(), on `stream` (a
 * cudaStream_t; NULL = a private stream), and load its state.  The next
 * update of the loaded model equals the next update the saved model would
 * have run.  DASH_EINVAL for a missing, truncated or corrupted file (bad
 * magic, version, sizes or checksum); allocation errors as dash_init(). */
dash_status dash_load(const char *path, void *stream, dash_model **out);

/* Reconstruction errors of the last update's new data with the updated
 * factors, from a second read of its rows (the paper's slice-level and
 * tensor-level reconstruction errors, Definitions 1-2, also its local error
 * of §4.1):
 *   se_k = Σ |X_k,new − X̂_k,new| / (I_k,new·J),  te = mean of se_k over the
 *   slices that received rows (ascending slice order),
 * with X̂_k,new = U_k,new S_k Vᵀ (mode P) or Q_k,new H S_k Vᵀ (mode Q), plus the
 * batch fitness of dash_fitness() computed from the direct residual.  Any
 * output may be NULL; se, if given, has se_len >= dash_num_slices() entries
 * and receives NaN for slices without new rows.  The rows are read where the
 * update read them: call it before staging anything new (DASH_ESTATE after
 * an append) and, for dash_update_device(), while the caller's X is still
 * valid.  Synchronises the stream. */
dash_status dash_local_errors(dash_model *m, double *te, double *fit_direct, double *se,
                              int64_t se_len);

/* Reconstruction error of any rows against the factors as they are now (the
 * paper's global error of §4.1 when the rows are the whole accumulated
 * tensor; Definitions 1-2 use the same residual):
 *   sq_err = Σ_i ||x_i − x̂_i||²,  sq_x = Σ_i ||x_i||²,  abs_err = Σ_i |x_i − x̂_i|_1
 * with x̂_i = u_i S_k Vᵀ (mode P) or u_i H S_k Vᵀ (mode Q).  Segment s covers
 * rows row_ptr[s]..row_ptr[s+1]-1 (row_ptr[0] = 0, ascending; host array)
 * and belongs to slice slice_ids[s] (host array, 0 <= id < the slice count).
 * X (device, input_dtype, row-major N×J) holds the rows and `rows` (device,
 * FP64, row-major N×R) their factor rows: U_k rows in mode P, Q_k rows in
 * mode Q, as the updates that saw them produced them (dash_new_rows).  Any
 * output may be NULL.  DASH_EINVAL for bad segments; synchronises the stream. */
dash_status dash_rows_error(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                            const int64_t *row_ptr, const void *X, const double *rows,
                            double *sq_err, double *sq_x, double *abs_err);

/* Wait for all work issued on the model's stream. */
dash_status dash_sync(dash_model *m);

/* Device memory (serving admission; the paper has no counterpart).
 * dash_config_bytes(): the device and pinned host bytes dash_init would
 * allocate for *cfg (each allocation rounded up to 512 bytes), computed
 * without allocating anything; DASH_EINVAL (and no sizes) for a config
 * dash_init would reject.  dash_device_bytes(): the device bytes the handle
 * owns (0 for NULL); the same figure as dash_config_bytes() for its config.
 * Either pointer may be NULL. */
dash_status dash_config_bytes(const dash_config *cfg, int64_t *device_bytes, int64_t *host_bytes);
int64_t dash_device_bytes(const dash_model *m);

/* Non-blocking completion test: *idle = 1 when every copy and kernel the
 * model has issued (its stream and its copy streams) has finished, else 0.
 * Never waits.  DASH_ECUDA if a stream reports an error. */
dash_status dash_query(const dash_model *m, int32_t *idle);

/* Per-update device time of the last dash_update (CUDA events, ms). */
dash_status dash_last_update_ms(const dash_model *m, float *ms);

/* Kernel accounting.  dash_launch_count(): kernels the library has launched
 * on this model since dash_init.  With profiling on, every launch is
 * bracketed by CUDA events on the model's stream and its device time is
 * accumulated per kernel kind (enabling resets the counters).
 * dash_profile_enable(): 0 off, 1 the per-launch events, 2 the events plus
 * in-kernel phase clocks of the streaming and slice-finish kernels (extra
 * work inside the kernels: for breakdowns, not for timing); DASH_EINVAL
 * otherwise.
 * dash_profile_get() reads kind i < dash_profile_kinds(): its name, the
 * launches and the total milliseconds since profiling was enabled; it
 * synchronises the stream.  *name points to static storage. */
int64_t dash_launch_count(const dash_model *m);

/* Numerical diagnostics since dash_init: bounded device waits that timed out,
 * and per-slice solves that left the mixed-precision fast path (a singular
 * map in Lemma 1 or an FP32 factor that was not trustworthy) for the FP64
 * pseudo-inverse.  Synchronises the stream. */
dash_status dash_counters(const dash_model *m, int64_t *timeouts, int64_t *fallbacks);
dash_status dash_profile_enable(dash_model *m, int32_t on);
int32_t dash_profile_kinds(void);
dash_status dash_profile_get(const dash_model *m, int32_t i, const char **name,
                             int64_t *launches, double *total_ms);

/* How the last update's batch was planned (diagnostics and roofline
 * accounting; the paper has no counterpart).  Mode P: rows and slices
 * finished by the fused row kernel's tiles (single-segment slices of at most
 * 256 rows), its tile count, rows of larger or split slices taken by the
 * chunked path, and rows of the general kernels (batches the fused path does
 * not take).  Mode Q: every row is a general row.  Any pointer may be NULL.
 * DASH_ESTATE before the first update. */
dash_status dash_last_plan(const dash_model *m, int64_t *tile_rows, int64_t *tile_slices,
                           int64_t *tiles, int64_t *chunk_rows, int64_t *general_rows);

/* Row pipeline of a mode-P update with FP32 input and DASH_PREC_F16X3
 * products (the paper has no counterpart: all compute Algorithm 1's P2-P7
 * on the same rows, in different kernels).
 *   DASH_ROWS_FUSED  tiles of single-segment slices (at most 256 new rows)
 *                    in one fused row kernel; other slices in row chunks.
 *   DASH_ROWS_SPLIT  every slice in row chunks: X·Q_V and the F increment
 *                    (Eq. 20) as two streaming tensor-core passes over X,
 *                    the per-slice work (P4, P6, P7) in between.  The X·Q_V
 *                    pass runs on tcgen05 MMAs fed by TMA (3-term TF32
 *                    split) where the shape allows it (J % 4 == 0, J <= 512,
 *                    R <= 32, 16-byte aligned rows), else as warp-level MMAs.
 *   DASH_ROWS_SPLIT_WARP  the same split pipeline with warp-level MMAs
 *                    (FP16 split) for both passes.
 *   DASH_ROWS_AUTO   the library's choice (currently DASH_ROWS_SPLIT).
 * Takes effect at the next update; other paths ignore it.  DASH_EINVAL for
 * an unknown value. */
enum { DASH_ROWS_AUTO = 0, DASH_ROWS_FUSED = 1, DASH_ROWS_SPLIT = 2, DASH_ROWS_SPLIT_WARP = 3 };
dash_status dash_set_row_path(dash_model *m, int32_t path);

/* Bounded device waits (the paper has no counterpart).  Every wait of the
 * streaming kernels on their copy pipeline gives up after a limit; the
 * update is then dropped by its own kernels: the ones that write the state
 * (c_k, D_k, W, F, G, V, VᵀV) see the flag and leave it as it was.  The next
 * synchronising call (dash_sync, a getter, or the planning of the next
 * update) returns DASH_ETIMEOUT once; the slice count returns to its value
 * before the dropped update, the dropped batch is gone, and the model stays
 * usable.
 * dash_set_wait_limit(): the limit of the tcgen05 streaming kernels, in SM
 * clock cycles (default 2·10⁹, about a second; the warp-level kernels keep
 * that default).  DASH_EINVAL below 1000.
 * dash_inject_wait_fault(): a test hook: in the next update, the first
 * thread block of the tcgen05 X·Q_V pass never issues the copy of its first
 * stage, so that its wait runs out.  DASH_ESTATE when this configuration has
 * no such pass (mode Q, FP64 or FP32 products, shapes it does not take). */
dash_status dash_set_wait_limit(dash_model *m, int64_t cycles);
dash_status dash_inject_wait_fault(dash_model *m);

/* Launch each update (dash_update, dash_update_device) as one CUDA graph
 * (the paper has no counterpart: the same kernels with the same arguments,
 * submitted at once).  The update's launch sequence is captured from the
 * model's stream; while its topology matches the previous update's (the same
 * kernels in the same order, as for batches of similar shape) the captured
 * arguments update the instantiated graph, otherwise it is instantiated
 * anew.  Off by default; ignored while profiling is on.  Results are
 * bit-identical either way.  dash_graph_stats() counts instantiations and
 * in-place updates (either pointer may be NULL).  Synchronises the stream. */
dash_status dash_set_graph(dash_model *m, int32_t on);
dash_status dash_graph_stats(const dash_model *m, int64_t *instantiations, int64_t *updates);

/* Autotuning of the X·Q_V pass (the paper has no counterpart: a choice
 * between kernels that compute the same bits).  With it on (the default),
 * the first mode-P update that runs the tcgen05 X·Q_V pass runs every
 * variant once and then times it on its own batch (the resident-Q_V kernel at each ring depth from
 * 2 to the deepest that fits, then the kernel that streams the Q_V slabs
 * with each stage), keeps the fastest for the rest of the model's life and
 * synchronises the stream once.  Skipped while graph updates are on (the
 * first update after they are turned off tunes).  Results are bit-identical whichever variant runs.
 * dash_autotune_result(): candidates timed (0 before tuning), the index of
 * the one kept (-1 before), whether the kept kernel is the resident-Q_V one,
 * its ring depth, and the candidates' times in ms (ms: 8 floats; unused
 * entries 0).  Any pointer may be NULL.  DASH_EINVAL for a bad switch. */
dash_status dash_set_autotune(dash_model *m, int32_t on);
dash_status dash_autotune_result(const dash_model *m, int32_t *n_candidates, int32_t *chosen,
                                 int32_t *resident, int32_t *ring, float *ms);

/* Measured FP64 FMA rate of the current device (FMAs per second; one FMA is
 * two flops): independent FMA chains on every SM, best of three timed runs
 * after a warm-up.  The FP64-product path and the per-slice R×R solves are
 * bound by this pipe; it is the denominator of their roofline.  Allocates a
 * few bytes (the paper has no counterpart).  DASH_ECUDA if the device
 * cannot be used. */
dash_status dash_measure_fp64_fma(double *fma_per_second);

/* Allocation-free F increment.  (The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory.)
 *
 * Computes F_inc = Σ_k X_k,newᵀ U_k,new S_k — the new-data term that
 * dash_update() adds to λF — with FP32 products and an FP64 sum, for callers
 * that may not call cudaMalloc or let a library call it: code under a host
 * framework whose memory manager owns the whole device, serving loops where
 * an allocation's implicit device synchronisation would stall work in
 * flight, and processes whose device footprint is fixed at start-up.
 *
 * All pointers are device pointers owned by the caller: X (N×J FP32,
 * row-major), U (N×R FP32, the rows' U_k,new), seg_row (n_seg+1 ascending
 * row offsets from 0) and seg_slice (n_seg slice ids) describing which slice
 * each row belongs to, W (rows of W for every id in seg_slice, FP64, K×R),
 * and the output F_inc (J×R FP64).  Work is queued on `stream` (a
 * cudaStream_t; NULL = the default stream) and the call returns without
 * waiting.
 *
 * Nothing is allocated: per-block partial sums go to one static device
 * array of 2^21 floats (8 MiB) that every GPU loading this library holds
 * until the process exits.  J·R above 2^21 returns DASH_ENOMEM; bad
 * arguments DASH_EINVAL; a failed lookup or launch DASH_ECUDA.  A call on a
 * stream that is not being captured looks that array's device address up
 * (with the device current) and caches it, so a context created anew after
 * cudaDeviceReset is followed; a call on a stream under capture uses the
 * cached address: make the first call on each device before any capture
 * (else DASH_ECUDA).  Calls share the array, so calls that overlap on the
 * GPU race; serialise them (e.g. one stream).  Each call writes every
 * partial it reads, so what an earlier call left there is never used. */
dash_status dash_f_increment_noalloc(const float *X, const float *U, int64_t N, int32_t J,
                                     int32_t R, const int64_t *seg_row, const int32_t *seg_slice,
                                     int64_t n_seg, const double *W, double *F_inc,
                                     void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DASH_H */
