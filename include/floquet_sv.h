/*
 * floquet_sv.h -- C ABI of the GB300 state-vector simulator for driven spin
 * chains (arXiv 2111.08044, "Simulation of quantum many-body dynamics with
 * Tensor Processing Units: Floquet prethermalization").
 *
 * The library evolves the full 2^L complex amplitude vector of an open chain
 * of L spin-1/2 sites by repeated application of a Floquet unitary,
 * |psi(nT)> = U_F^n |psi(0)> (Eq. 3), and measures the energy density
 * <psi|H0|psi>/L once per period (Eq. 10 with H0 the time-averaged
 * Hamiltonian of Eq. 7).
 *
 * Conventions shared by every call:
 *   - Site i is bit i of the amplitude index (little-endian).  A two-site
 *     operator on bond (i, i+1) is a row-major 4x4 matrix with local index
 *     r = 2*b_i + b_{i+1} (site i is the high bit), as in the contraction
 *     U_{b7 b8 alpha beta} of Eq. 2.
 *   - |0> is spin up: Z|0> = +|0>.
 *   - One period: K Trotter steps, each all gates on bonds of parity
 *     `first_layer` then all gates on the other parity (the two-layer
 *     brickwork of Eq. 4), every gate exp(-i tau h_b) (Eq. 5) with tau = T/K
 *     and h_b = J Z_i Z_{i+1} + c_x(i) X_i + c_x(i+1) X_{i+1}
 *                             + c_z(i) Z_i + c_z(i+1) Z_{i+1},
 *     where each bond gives each of its sites h/2 of the on-site fields,
 *     except that an open end site receives edge_field_weight * h from its
 *     one bond; then the kick exp(-i theta sum_i X_i).
 *   - H0 = sum_b h_b (Eq. 7).  Reported energy densities are those of the
 *     normalised state, <psi|H0|psi> / (L <psi|psi>); the squared norm, which
 *     drifts from 1 only by rounding, is reported beside them.
 *   - Status: every call returns SV_OK (0) or a negative SV_E* code; no
 *     exception or abort crosses this boundary.  sv_last_error() gives text.
 *   - Memory: the state buffer belongs to the caller (device memory, e.g. a
 *     torch tensor).  The library allocates only small device buffers
 *     (gate tables, fused unitaries, reduction partials, the energy ring).
 *   - Streams: every launch goes to the stream given at sv_create, in call
 *     order.  Calls with host outputs synchronise that stream before
 *     returning.
 */
#ifndef FLOQUET_SV_H
#define FLOQUET_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SV_OK 0
#define SV_EINVAL (-1)      /* bad argument (size, range, null pointer) */
#define SV_ENOMEM (-2)      /* a library allocation failed */
#define SV_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define SV_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define SV_ESTATE (-5)      /* calls made in the wrong order */
#define SV_EUNSUPPORTED (-6) /* valid request this build does not implement */

/* state precision */
#define SV_C64 0  /* complex64 amplitudes, FP32 arithmetic, FP64 reductions */
#define SV_C128 1 /* complex128 amplitudes, FP64 arithmetic (check mode) */
#define SV_DF64 2 /* double-float check mode: each real number is an unevaluated
                     sum hi + lo of two FP32 values (about 48 significant bits),
                     16 bytes an amplitude (hi re, lo re, hi im, lo im), FP32
                     arithmetic (error-free sums and FMA products); plain mode
                     only.  Read and written as complex128 by sv_get_state /
                     sv_set_state. */

/* evolution form */
#define SV_MODE_PLAIN 0 /* one kernel pass per two-qubit gate */
#define SV_MODE_BLOCK 1 /* fused n-qubit blocks on the tensor cores */
#define SV_MODE_MULTIGATE 2 /* many gates per pass on a shared-memory tile (CUDA cores) */

/* arithmetic of the block form */
#define SV_SPLIT_BF16X3 0 /* tensor cores: 3 exact bf16 digits per operand, exact level-0 sum */
#define SV_SPLIT_FP32 1   /* FP32 CUDA-core block apply (reference form) */

typedef struct sv_ctx sv_ctx;

/* Parameters of the driven chain and of the evolution form. */
typedef struct sv_floquet_params {
  double J;                 /* Z Z coupling */
  double hx;                /* transverse field */
  double hz;                /* longitudinal field */
  double T;                 /* Floquet period */
  double theta;             /* kick angle: kick = exp(-i theta sum X) */
  double edge_field_weight; /* field share of an open end site (0.5: uniform) */
  int32_t K;                /* Trotter steps per period, >= 1 */
  int32_t first_layer;      /* 0: bonds (0,1),(2,3),.. first; 1: odd bonds first */
  int32_t mode;             /* SV_MODE_PLAIN, SV_MODE_BLOCK or SV_MODE_MULTIGATE */
  int32_t block_n;          /* block width n for SV_MODE_BLOCK (2..7); 0 = default */
  int32_t split;            /* SV_SPLIT_* (block mode) */
  int32_t renorm_every;     /* rescale psi to unit norm at the start of every this
                               many-th period (folded into its first pass, using the
                               FP64 norm measured at the end of the previous period);
                               0 = never */
  int64_t n_period_params;  /* > 0: theta_p / hx_p give one value per period */
  const double *theta_p;    /* host, length n_period_params, or NULL */
  const double *hx_p;       /* host, length n_period_params, or NULL */
  int32_t inverse;          /* 1: every period applies U_F^dagger instead of U_F (the
                               kick undone first, then the gates in reverse order,
                               each replaced by its adjoint), as in the echo of
                               Sec. V; energies are measured at the end of each
                               inverse period.  Needs n_period_params = 0. */
  const double *h_bonds;    /* NULL: the driven Ising chain above.  Otherwise host,
                               (L-1) x 16 complex (row-major 4x4, local index
                               r = 2 b_i + b_{i+1}; site i the high bit): the
                               Hermitian bond terms H_b of a general two-site chain
                               (the random circuits of Sec. III.A), whose gates are
                               exp(-i (T/K) H_b) and whose energy observable is
                               sum_b H_b (Eq. 7); J, hx, hz and edge_field_weight
                               are then unused.  sv_evolve does not measure such a
                               chain per period (its energy and norm outputs are
                               NaN); sv_energy_moments / sv_expect_energy measure
                               it on demand.  Needs n_period_params = 0 and
                               renorm_every = 0. */
} sv_floquet_params;

/* Library version (an integer that grows with the ABI). */
int sv_version(void);

/*
 * Create a context on CUDA device `device` for amplitudes of the given
 * precision (SV_C64, SV_C128 or SV_DF64; SV_DF64 contexts have no
 * sv_energy_moments, overlaps, sv_init_pairs, sv_adjoint, nor measurement of
 * general chains: those return SV_EUNSUPPORTED).  `cuda_stream` is a cudaStream_t (NULL:
 * the legacy default stream).  *out receives the handle; free it with
 * sv_destroy.  Errors: SV_EINVAL (bad precision / null out), SV_ECUDA (no
 * such device), SV_ENOMEM.
 */
int sv_create(sv_ctx **out, int device, int precision, void *cuda_stream);

/*
 * Attach the caller's device buffer that holds the state: at least
 * 8*2^L bytes (SV_C64) or 16*2^L bytes (SV_C128, SV_DF64), 256-byte aligned,
 * interleaved (re, im).  The caller keeps ownership and must keep it alive
 * while the context uses it.  Errors: SV_EINVAL (null or misaligned).
 */
int sv_attach_state(sv_ctx *ctx, void *dev_ptr, size_t bytes);

/*
 * Write the product state psi_x = prod_i s_i[b_i(x)] (a product initial
 * state, cf. Eq. 9) into the attached buffer.  product_state: host array of
 * 4*L doubles, per site (re a, im a, re b, im b) with a the |0> and b the
 * |1> component; the library normalises each site.  Resets the period
 * counter to 0.  L: 2..34 (SV_C64), 2..33 (SV_C128, SV_DF64).  Errors: SV_EINVAL
 * (L out of range, buffer too small, zero spinor), SV_ESTATE (no buffer).
 */
int sv_init(sv_ctx *ctx, int L, const double *product_state);

/*
 * Dimer-product initial state psi = (x)_k phi_k over the site pairs
 * (2k, 2k+1), k = 0..L/2-1 (L even): the product of two-site ground states
 * that starts the evolutions of Sec. III.B (Eq. 9).  pair_states: host,
 * (L/2) x 4 complex = 4L doubles, local index r = 2 b_{2k} + b_{2k+1} (the
 * lower site the high bit, as for the bond terms); each pair's vector is
 * normalised.  Resets the period counter like sv_init.  Errors: SV_EINVAL,
 * SV_ESTATE, SV_ECUDA.
 */
int sv_init_pairs(sv_ctx *ctx, int L, const double *pair_states);

/* <phi|psi> with the dimer-product state phi of pair_states (as for
 * sv_init_pairs); FP64.  Errors: SV_EINVAL, SV_ESTATE, SV_ECUDA. */
int sv_overlap_pairs(sv_ctx *ctx, const double *pair_states, double *overlap_re,
                     double *overlap_im);

/*
 * Build the period: FP64 bond gates exp(-i tau h_b) (Eq. 5), kick folding
 * into the last gate on each site, and, in block mode, the fusion of gates
 * into n-qubit block unitaries (the >= 7-qubit operators of Sec. II, built
 * here in FP64).  Uploads everything the evolution needs.  Requires
 * sv_init.  Per-period parameters (n_period_params > 0) are supported in
 * plain mode only.  Errors: SV_EINVAL, SV_ESTATE, SV_EUNSUPPORTED,
 * SV_ENOMEM, SV_ECUDA.
 */
int sv_build_floquet(sv_ctx *ctx, const sv_floquet_params *p);

/*
 * Apply `periods` periods (Eq. 3).  After each period the energy density
 * <psi|H0|psi>/(L <psi|psi>) and <psi|psi> are recorded; energy_out / norm_out (host,
 * length `periods`, either may be NULL) receive them.  With per-period
 * parameters the period counter must stay below n_period_params.
 * Errors: SV_EINVAL, SV_ESTATE, SV_ECUDA, SV_ETIMEOUT (a tensor-core pass
 * gave up a bounded wait; reported when the call synchronises, i.e. when
 * energy_out or norm_out is given).
 */
int sv_evolve(sv_ctx *ctx, int64_t periods, double *energy_out, double *norm_out);

/*
 * sv_evolve without the CUDA graph, for measurement: every kernel launch of
 * a period is bracketed by CUDA events on the context's stream, and
 * pass_ms[k] (host, length launches_per_period from sv_pass_info, nullable)
 * accumulates the duration of launch k of the period over all periods, in
 * milliseconds.  Results are identical to sv_evolve.  Errors as sv_evolve.
 */
int sv_evolve_profiled(sv_ctx *ctx, int64_t periods, double *energy_out,
                       double *norm_out, double *pass_ms);

/*
 * Energy density <psi|H0|psi>/(L <psi|psi>) (Eq. 10 per site) and <psi|psi> of the current
 * state (host outputs; either may be NULL).  Errors: SV_ESTATE, SV_ECUDA.
 */
int sv_expect_energy(sv_ctx *ctx, double *energy_density, double *norm2);

/*
 * Energy moments of the current state (Sec. III.B): energy = E = <H0> and
 * sigma_e = sqrt(<H0^2> - E^2) of the normalised state (Eq. 10, Eq. 11; the
 * energy itself, not per site), and norm2 = <psi|psi>; any output may be
 * NULL.  <H0^2> = |H0 psi|^2 is accumulated with H0 psi formed amplitude by
 * amplitude from each amplitude's L bit-flip neighbours: no second state is
 * held, and the state is read about L + 1 times.  Errors: SV_ESTATE,
 * SV_ECUDA.
 */
int sv_energy_moments(sv_ctx *ctx, double *energy, double *sigma_e, double *norm2);

/*
 * Overlap <phi|psi> of the current state with the product state phi of
 * `spinors` (host, L*4 doubles as for sv_init; each site's spinor is
 * normalised): with phi the state sv_init started from, after P periods
 * and P inverse periods (sv_floquet_params.inverse) this is the echo
 * overlap of Sec. V, whose error is |1 - <psi(0)|psi'(0)>|.  Computed in FP64
 * from a table of the low sites times a table of the others.  Errors:
 * SV_EINVAL, SV_ESTATE, SV_ECUDA.
 */
int sv_overlap_product(sv_ctx *ctx, const double *spinors, double *overlap_re,
                       double *overlap_im);

/* Scale psi to unit norm (FP64 norm); *norm2_before (nullable) gets the
 * squared norm it had.  Errors: SV_ESTATE, SV_ECUDA. */
int sv_renormalize(sv_ctx *ctx, double *norm2_before);

/*
 * Reverse-mode gradient of the final energy density f = <psi_P|H0|psi_P>/L
 * after P = `periods` periods with respect to the per-period kick angles
 * theta_p and fields hx_p of those periods (p = 0..P-1; plain mode, built
 * with n_period_params >= P, period counter at 0).  Starting from the
 * current state it evolves P periods forward without storing states, seeds
 * lambda = (H0/L) psi_P, and walks the gates backwards, un-applying each on
 * psi and lambda while accumulating 2 Re <lambda| dG G^dagger |psi>.  On
 * return the state buffer holds psi back at its starting point up to
 * rounding and the counter is 0.  grad_theta / grad_hx: host, length P
 * (nullable).  energy_density (nullable): f.  Needs 2x the state memory for
 * lambda, allocated by the library.  Errors: SV_EINVAL (periods outside
 * 1..n_period_params), SV_ESTATE, SV_ENOMEM, SV_ECUDA, SV_EUNSUPPORTED.
 */
int sv_adjoint(sv_ctx *ctx, int64_t periods, double *grad_theta, double *grad_hx,
               double *energy_density);

/* Copy the state, natural layout, to `host_dst`: host memory or device
 * memory of the context's device (bytes >= state size).  SV_C64 and SV_C128
 * copy the amplitudes as held; SV_DF64 writes complex128 (hi + lo, exact in
 * FP64), converted on the device through a 64 MiB buffer the call
 * allocates.  Errors: SV_EINVAL, SV_ESTATE, SV_ECUDA. */
int sv_get_state(sv_ctx *ctx, void *host_dst, size_t bytes);

/* Copy a state from host memory into the attached buffer (for checkpoint
 * resume); sets the period counter.  SV_DF64 reads complex128 and keeps
 * each part as the nearest float plus the nearest float to the remainder
 * (relative error at most 2^-48).  Errors as sv_get_state. */
int sv_set_state(sv_ctx *ctx, const void *host_src, size_t bytes, int64_t period);

/*
 * Checkpoints of long evolutions (the paper runs more than 1e5 periods,
 * Sec. IV): the state and the period counter in one file.  Layout,
 * little-endian: bytes 0-7 "FLQSVCK1"; int32 L; int32 precision; int64
 * period counter; uint64 payload bytes; uint64 checksum of the payload;
 * uint64 checksum of bytes 0-39; then the 2^L amplitudes in the natural
 * layout (interleaved re, im, complex64 or complex128; SV_DF64: the
 * double-float words as held, hi re, lo re, hi im, lo im).  Checksums:
 * FNV-1a (64-bit basis and prime) over little-endian 64-bit words.
 *
 * sv_save writes the attached state (stream-ordered after earlier calls)
 * and the counter to `path`, through a 64 MiB pinned host buffer the call
 * allocates and frees.  Errors: SV_EINVAL (null path, file not writable),
 * SV_ESTATE (no state), SV_ENOMEM, SV_ECUDA.
 *
 * sv_load reads a checkpoint into the attached state buffer (which must
 * hold it) and sets L and the period counter as sv_init / sv_set_state
 * would; a built evolution stays valid when its L matches.  The precision
 * must be the context's.  On a truncated file or a checksum mismatch it
 * returns SV_EINVAL with the amplitudes overwritten but L and the counter
 * unchanged.  Errors: SV_EINVAL, SV_ESTATE, SV_ENOMEM, SV_ECUDA.
 *
 * sv_checkpoint_info checks a file (header, payload checksum and size)
 * without a GPU and reports its L, precision and period (each nullable).
 * Errors: SV_EINVAL.
 */
int sv_save(sv_ctx *ctx, const char *path);
int sv_load(sv_ctx *ctx, const char *path);
int sv_checkpoint_info(const char *path, int *L, int *precision, int64_t *period);

/*
 * Layout of the state between sv_evolve calls.  A block plan may start its
 * periods at a window off site 0; an evolution then relabels the state into
 * that window's layout first and its last period hands back the natural
 * layout, one extra pass per call.  With keep_period_layout = 1 the state
 * stays in the period layout after sv_evolve / sv_evolve_profiled (callers
 * evolving one period per call save that pass); every call that reads the
 * state (sv_get_state, sv_expect_energy, sv_energy_moments, the overlaps,
 * sv_renormalize, sv_adjoint, sv_save) and sv_build_floquet bring it back to
 * the natural layout first, and calls that write the state set it natural.
 * Meanwhile the attached buffer, read directly, holds the amplitudes in the
 * period layout (window of the plan's first pass on bits 0..n-1).
 * keep_period_layout = 0 (the default) restores the natural layout at once.
 * Errors: SV_EINVAL, SV_ECUDA.
 */
int sv_set_layout_policy(sv_ctx *ctx, int keep_period_layout);

/* Periods applied since sv_init / sv_set_state / sv_load. */
int64_t sv_period_counter(const sv_ctx *ctx);

/*
 * Kernel passes over the state per period and two-qubit gates per period
 * of the built evolution (for throughput accounting).  Errors: SV_ESTATE.
 */
int sv_pass_info(const sv_ctx *ctx, int *passes_per_period, int *gates_per_period,
                 int *launches_per_period);

/*
 * The evolution form sv_build_floquet chose: *tensor_cores = 1 when block
 * passes run on the tensor cores (tcgen05, n = 6 windows on chains of at
 * least 13 sites), 0 for the CUDA-core block pass or the plain form;
 * *block_n = window width (0 in plain mode).  Errors: SV_ESTATE.
 */
int sv_form_info(const sv_ctx *ctx, int *tensor_cores, int *block_n);

/* Bytes the last sv_build_floquet copied host -> device (gate tables, fused
 * unitaries, tensor-core operands).  Errors: SV_ESTATE. */
int sv_build_bytes(const sv_ctx *ctx, size_t *h2d_bytes);

/* Text of the last error on this context ("" if none). Never NULL. */
const char *sv_last_error(const sv_ctx *ctx);

/* Release the context and its library buffers (not the state buffer). */
void sv_destroy(sv_ctx *ctx);

/*
 * Energy density <psi|H0|psi>/(L <psi|psi>) and squared norm of a chain
 * state, for callers that cannot allocate device memory (for example code
 * that runs while a stream is being captured with a memory pool it does not
 * own, or a process whose device memory all belongs to an outside
 * allocator).  The paper has no counterpart: it is a deployment variant of
 * the measurement that sv_expect_energy makes.
 *
 *   psi_dev     device pointer to the 2^L amplitudes (complex64 or
 *               complex128 by `precision`), natural layout; read only.
 *   p           host parameters of H0 (J, hx, hz, edge_field_weight; the
 *               other fields must be valid as for sv_build_floquet).
 *   out_dev     device pointer to 2 doubles, written on `cuda_stream`:
 *               out_dev[0] energy density, out_dev[1] <psi|psi>.
 *   cuda_stream cudaStream_t the launches go to (NULL: legacy stream).
 *
 * Allocates nothing: its reduction scratch is a fixed 288 KiB device array
 * of the library, held on every device that loads the library until the
 * process exits; it supports L <= 34 (complex64) / 33 (complex128).  The
 * first call on a device looks that array up on the current device, so
 * make the first call before any stream capture.  Every call reuses the
 * same array (zeroing it first), so calls that overlap on the GPU race: do
 * not run two at once.  It measures the driven Ising chain's H0 only: a
 * chain given by general bond terms (p->h_bonds set; its observable is
 * sum_b H_b, Eq. 7) is refused, use sv_expect_energy for it.  Returns
 * without synchronising.  Errors: SV_EINVAL (null pointer, bad precision,
 * L beyond the limit, invalid parameters, p->h_bonds set), SV_ECUDA
 * (symbol lookup or launch failed).
 */
int sv_energy_noalloc(const void *psi_dev, int L, int precision,
                      const sv_floquet_params *p, double *out_dev, void *cuda_stream);

/* ------------------------------------------------------------------ host
 * Host-side builders, callable without a GPU, exposed for inspection and
 * testing of the period construction.
 */

/*
 * FP64 bond gates exp(-i tau h_b) (Eq. 5) for b = 0..L-2 (gates_out:
 * (L-1)*32 doubles, row-major complex 4x4) and the kick exp(-i theta X)
 * (kick_out: 8 doubles).  Either output may be NULL.  Errors: SV_EINVAL.
 */
int sv_host_bond_gates(int L, const sv_floquet_params *p, double *gates_out,
                       double *kick_out);

/*
 * The period as the library applies it in plain mode: gates in application
 * order with the kick folded into the last gate on each site.  bonds_out
 * (int[*n_gates]) and mats_out (32 doubles per gate) may be NULL to query
 * the count; *n_gates is in/out (capacity in, count out).  Errors: SV_EINVAL.
 */
int sv_host_period_gates(int L, const sv_floquet_params *p, int *n_gates,
                         int *bonds_out, double *mats_out);

/*
 * Block-mode fusion plan for one period with blocks of n sites.
 * *n_passes is in/out (capacity in, count out).  For pass k:
 * window_lo[k] is the first site of its n-site window, gate_count[k] the
 * number of two-qubit gates fused into it, and, if unitaries_out is not
 * NULL, unitaries_out + k*2*4^n holds the fused 2^n x 2^n unitary (row-major
 * complex, local bit j = site window_lo + j).  Errors: SV_EINVAL.
 */
int sv_host_fusion_plan(int L, const sv_floquet_params *p, int n, int *n_passes,
                        int *window_lo, int *gate_count, double *unitaries_out);

/*
 * The operand a block pass applies in place of pass `pass`'s fused unitary
 * (see sv_host_fusion_plan): the fused 2^n x 2^n unitary of the window as
 * the pass's number format represents it, chosen entry by entry between the
 * two representable values bracketing the exact entry so that the matrix is
 * as close to unitary as the format allows (the same operand is applied
 * every period, so a defect U^H U - I would change the norm by the same
 * amount every period).  split = SV_SPLIT_FP32: the CUDA-core pass's FP32
 * entries; SV_SPLIT_BF16X3 (n = 6): the value of the tensor-core pass's
 * three digits u = 2^-7 (u0 + u1/256 + u2/65536).  operand_out: 2*4^n
 * doubles, row-major complex.  Errors: SV_EINVAL.
 */
int sv_host_pass_operand(int L, const sv_floquet_params *p, int n, int pass, int split,
                         double *operand_out);

/*
 * Block-mode tile layout of each pass (the relabel of Sec. II's qubit
 * swaps folded into the pass's write; n < L).  *n_passes is in/out as
 * above.  For pass k, any output may be NULL:
 *   tile_a[k]                the first state bit of the tile's row bits;
 *   sigma_out[13k + q]       the output tile bit of input tile bit q (window
 *                            bits q < n, then min(7, L - n) row bits; -1
 *                            past the tile);
 *   rows_out[7k + i]         for the tensor-core pass (n = 6, L >= 13), the
 *                            tile row bits held by TMEM lane bit i (an
 *                            invertible map over GF(2); 0 otherwise);
 *   store_wavefronts[k]      that pass's shared-memory wavefronts per warp
 *                            store of its relabelled write (2 = free of bank
 *                            conflicts; 0 if not a tensor-core pass);
 *   x_sites_out[k]           bit j set if the pass measures <X> of window
 *                            site window_lo + j (each site once per period,
 *                            in the pass holding its last gate);
 *   staging_out[13k + o]     tensor-core pass: the bit of the staging tile
 *                            that holds output tile bit o (o for the natural
 *                            order; bits 0-3 always stay in place).
 * Errors: SV_EINVAL.
 */
int sv_host_block_layout(int L, const sv_floquet_params *p, int n, int *n_passes,
                         int *tile_a, int *sigma_out, unsigned char *rows_out,
                         int *store_wavefronts, int *x_sites_out,
                         unsigned char *staging_out);

/* Host only, no device work: the TMA store view of tensor-core pass `pass`
 * (n = 6, L >= 13) of the fusion plan for (L, *p) -- the layout the pass's
 * 64 KiB staging tile is written back through.  Outputs:
 *   *rank                     3 to 5 (dimension 0 plus one per run of the
 *                             staging order);
 *   dims[5], box[5]           extents in amplitudes (8-byte elements) of
 *                             the view and of the stored box (1 past rank);
 *   strides[4]                byte strides of dimensions 1..rank-1;
 *   coord[4]                  tile t = tlo + 2^(a-6) thi is stored at
 *                             coordinate tlo << coord[1] of dimension
 *                             coord[0] and thi << coord[3] of dimension
 *                             coord[2], all other coordinates 0.
 * Staging element s (box order, dimension 0 fastest) of tile t lands at
 * amplitude sum_d (c_d + i_d) strides_d / 8.  Ownership: caller buffers.
 * Errors: SV_EINVAL (bad arguments, pass out of range, not a tensor-core
 * width). */
int sv_host_store_view(int L, const sv_floquet_params *p, int n, int pass, int *rank,
                       unsigned long long *dims, unsigned long long *strides, unsigned *box,
                       int *coord);

/* ------------------------------------------------------------------ batch
 * Many independent chains (each its own L, parameters and product state)
 * evolved together on one device.  Chains of up to 14 sites can stay in one
 * CTA's shared memory for a whole run (resident form); the others run the
 * plain, block or multi-gate forms.  One CUDA graph advances every chain by
 * a run of periods, the chains as independent branches (within a run a
 * chain's block periods may start off site 0; every run hands back the
 * natural layout).  Tensor-core chains of one L run as a group: each pass
 * of all of them is one launch over all their tiles, and each period's
 * energy reduces are one launch.  An autotuner times the forms that fit
 * each distinct L (the CUDA-core block form at its widths) on a few of its
 * chains and keeps the fastest (chain-periods per second).
 */
typedef struct sv_batch sv_batch;

#define SV_BATCH_AUTO (-1)      /* autotune per distinct L */
#define SV_BATCH_PLAIN 0        /* per-gate passes */
#define SV_BATCH_BLOCK_SIMT 1   /* fused windows on CUDA cores: n = 5..7 chosen by the
                                   autotuner, n = 6 when the form is forced */
#define SV_BATCH_BLOCK_TC 2     /* fused n = 6 windows on the tensor cores (L >= 13) */
#define SV_BATCH_RESIDENT 3     /* state in one CTA's shared memory (L <= 14) */
#define SV_BATCH_MULTIGATE 4    /* many gates per pass on a shared-memory tile */

/* Bytes of the state buffer for n_chains chains of sizes L[0..n_chains):
 * complex64 states back to back, each starting on a 256-byte boundary. */
size_t sv_batch_state_bytes(int n_chains, const int *L);

/*
 * Create a batch on `device` and initialise every chain's product state.
 * L: n_chains sizes (2..34); params: n_chains parameter sets (mode, split,
 * block_n and per-period arrays are ignored / must be absent); product_states:
 * the chains' spinors back to back (4 L_c doubles each, as sv_init);
 * state_dev: caller-owned device buffer of >= sv_batch_state_bytes bytes;
 * form: SV_BATCH_AUTO or one SV_BATCH_* form for every chain (a form a
 * chain cannot use falls back to SV_BATCH_PLAIN).  Errors: SV_EINVAL,
 * SV_ENOMEM, SV_ECUDA (*out is NULL on error).
 */
int sv_batch_create(sv_batch **out, int device, int n_chains, const int *L,
                    const sv_floquet_params *params, const double *product_states,
                    void *state_dev, size_t bytes, int form, void *cuda_stream);

/* Advance every chain by `periods`; energy_out / norm_out (nullable, host):
 * [n_chains][periods] row-major energy densities (normalised state) and
 * norms.  Errors: SV_EINVAL, SV_ECUDA, SV_ETIMEOUT. */
int sv_batch_evolve(sv_batch *b, int64_t periods, double *energy_out, double *norm_out);

/* The SV_BATCH_* form each chain runs (host array of n_chains). */
int sv_batch_forms(const sv_batch *b, int *form_out);

/* The block width n of each chain's form (host array of n_chains; 0 for
 * the plain, resident and multi-gate forms). */
int sv_batch_widths(const sv_batch *b, int *n_out);

const char *sv_batch_last_error(const sv_batch *b);
void sv_batch_destroy(sv_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* FLOQUET_SV_H */
