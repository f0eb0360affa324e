/*
 * vqnqs.h - C ABI of the GB300 (sm_103a) VQ-NQS local-energy library.
 *
 * The library evaluates the Vector-Quantized Neural Quantum State of
 * arXiv 2212.11296 and the variational-Monte-Carlo local energy
 *
 *     E_loc(s) = sum_{s'} H_{s s'} psi(s') / psi(s)             (Sec. 2, Eq. local-energy)
 *
 * for the spin-1/2 Heisenberg model H = J sum_<ij> S_i . S_j on an L x L
 * square lattice (Sec. 4), in the Marshall-rotated basis where psi > 0 and
 * the phase is zero (Sec. 4), or for the transverse-field Ising chain of
 * Sec. 4 (vqnqs_create_tfim).  psi(s) = sqrt(P(s)) with P an autoregressive
 * decoder transformer, one token per spin, whose blocks insert a vector
 * quantizer between the self-attention and its output projection (Sec. 3.1,
 * Eq. vq).  Per-location work whose quantized input was already seen is done
 * once per unique (row, code) key (Sec. 3.2) when VQNQS_REUSE is set.
 *
 * Conventions shared by every entry point
 *  - Spins: uint8 in {0 = down, 1 = up}, raster order p = y * L + x, one row
 *    of N = L * L bytes per sample.  Any configuration is accepted (S_z = 0 is
 *    not required).  Values other than 0/1 raise VQNQS_DEV_BAD_SPIN.
 *  - Array arguments named dev_* are DEVICE pointers owned by the caller;
 *    weights passed to vqnqs_create are HOST memory and are copied.
 *  - VQNQS_BF16 needs d_model % 64 == 0.
 *  - Calls that take a stream enqueue work on that cudaStream_t (NULL = legacy
 *    default stream) and return without synchronising; outputs are valid after
 *    the caller synchronises the stream.  They allocate nothing: all scratch
 *    lives in the caller's workspace (see vqnqs_workspace_bytes).
 *  - Every call returns a vqnqs_status; on failure vqnqs_last_error gives a
 *    message.  Errors detected inside kernels set bits of a device status word
 *    that vqnqs_get_stats reports; kernels never trap.
 *  - A context is used by one host thread at a time.
 *
 * Weight blob (float32, in this order; d = d_model, n_max = L * L):
 *   tok_emb[3][d] (token 0 down, 1 up, 2 begin-of-sequence), pos_emb[n_max][d],
 *   per layer: ln1_g[d] ln1_b[d] w_qkv[d][3d] b_qkv[3d] codebook[K][d]
 *              w_o[d][d] b_o[d] ln2_g[d] ln2_b[d] w_1[d][4d] b_1[4d]
 *              w_2[4d][d] b_2[d],
 *   lnf_g[d] lnf_b[d] w_head[d][2] b_head[2].
 * Matrices are row-major and multiply from the right (x @ w).
 */
#ifndef VQNQS_H
#define VQNQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vqnqs_ctx vqnqs_ctx;

typedef enum {
    VQNQS_OK = 0,
    VQNQS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad flag) */
    VQNQS_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    VQNQS_ERR_OOM = 3,        /* device allocation failed (vqnqs_create only) */
    VQNQS_ERR_WORKSPACE = 4,  /* workspace smaller than the one-sample minimum */
    VQNQS_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
    VQNQS_ERR_INTERNAL = 6
} vqnqs_status;

/* flags (bitwise or); 0 = plain full recompute in FP32 */
enum {
    VQNQS_REUSE = 1,       /* deduplicate per-location work by (row, code) keys (Sec. 3.2) */
    VQNQS_BF16 = 2,        /* BF16 tensor-core GEMMs with FP32 accumulation */
    VQNQS_INCREMENTAL = 4, /* with VQNQS_REUSE, local energies only: a connected configuration's
                              attention rows whose query is the sample's are corrected for the
                              changed keys only, and their codeword is taken from the sample's row
                              when a distance bound proves it unchanged (else searched).  Exact up
                              to rounding; the paper leaves attention dense (Sec. 3.2).  Needs
                              d_model in {32, 64, 128, 256, 512} and d_model / heads in {16, 32},
                              a multiple of d_model / 32. */
    VQNQS_BF16_SPLIT = 8   /* with VQNQS_BF16: every tensor-core product takes its operands as BF16
                              pairs x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and sums
                              hi.hi + hi.lo + lo.hi in FP32, three BF16 MMAs per product: the pair
                              holds x to 2^-17 relative (one BF16 value: 2^-9), so the GEMMs and
                              the attention carry FP32-grade error and the Eq. vq codeword choices
                              follow the exact ones except on rows whose relative distance gap is
                              within that error.  Local energies, log psi and codes; needs
                              d_model / heads in {16, 32}, at most 256 positions and no final
                              half-block (with VQNQS_INCREMENTAL: d_model / heads = 32 and
                              d_model in {128, 256}).  The sampler and the gradient ignore it. */
};

/* bits of the device status word */
enum {
    VQNQS_DEV_BAD_SPIN = 1,       /* a spin byte was not 0 or 1 */
    VQNQS_DEV_HASH_OVERFLOW = 2,  /* a dedupe probe ran past its bound */
    VQNQS_DEV_TIMEOUT = 4,        /* a bounded wait gave up */
    VQNQS_DEV_NONFINITE = 8       /* a row reached the codeword search with no finite distance (its
                                     values were not finite); it was given codeword 0 */
};

#define VQNQS_MAX_LAYERS 64

typedef struct vqnqs_stats {
    int64_t samples;                          /* samples processed since the last reset */
    int64_t configs;                          /* configurations evaluated (samples + connected ones) */
    int64_t rows;                             /* configs * N: token rows per layer */
    int64_t unique_rows[VQNQS_MAX_LAYERS + 1];/* sum over chunks of the unique per-location rows
                                                 feeding layer l (index l), and the head (index layers) */
    int64_t near_ties;                        /* code assignments with relative distance gap < 1e-6 */
    double flops_full;                        /* analytic FLOPs (2 per MAC) of full recompute */
    double flops_done;                        /* analytic FLOPs of the work actually executed */
    int32_t device_status;                    /* OR of VQNQS_DEV_* bits raised so far */
    int64_t active_rows;                      /* rows per layer whose attention and code were computed
                                                 (rows before a configuration's first exchanged site
                                                 reuse the sample's own rows) */
    int64_t attn_pairs;                       /* causal query-key pairs of those rows, per layer */
    /* VQNQS_INCREMENTAL, summed over layers: */
    int64_t inc_base_rows;                    /* samples' own rows (full attention, codeword certificate) */
    int64_t inc_patched_rows;                 /* rows whose attention was corrected for the changed keys */
    int64_t inc_certified_rows;               /* patched rows whose codeword was proved to be the sample's */
    int64_t inc_full_rows;                    /* rows whose attention was recomputed over all keys */
    int64_t inc_searched_rows;                /* rows given to the nearest-codeword search */
    int64_t inc_patch_pairs;                  /* (patched row, changed key) pairs, per head */
    int64_t inc_full_pairs;                   /* causal query-key pairs of the recomputed rows, per head */
    int64_t inc_whole_pairs;                  /* causal query-key pairs, per head, of the configurations
                                                 recomputed whole (rows from the first changed position) */
} vqnqs_stats;

/* Number of floats in the weight blob for the layout above. */
size_t vqnqs_num_params(int n_max, int layers, int d_model, int K);

/* Create a context.
 *   L        lattice side (sites N = L * L; 4 <= N <= 512)
 *   periodic 1 = periodic boundaries (2N bonds), 0 = open (2L(L-1) bonds)
 *   J        exchange coupling of H = J sum_<ij> S_i . S_j
 *   layers, d_model, heads, K   model shape: 1 <= layers <= VQNQS_MAX_LAYERS,
 *            32 <= d_model <= 1024 with d_model % 32 == 0, d_model / heads in
 *            {8, 16, 32}, 1 <= K <= 65535
 *   weights  HOST float32 blob of vqnqs_num_params(L*L, layers, d_model, K) values (copied)
 * The context owns device copies of the weights and of tables derived from
 * them (codebook projections through W_o, codebook norms, BF16 transposes).
 * Returns VQNQS_ERR_ARG / VQNQS_ERR_OOM / VQNQS_ERR_CUDA on failure (*out = NULL). */
int vqnqs_create(int L, int periodic, double J, int layers, int d_model, int heads, int K,
                 const float* weights, vqnqs_ctx** out);

/* Create a context for the transverse-field Ising chain of Sec. 4,
 *     H = -J sum_<ij> sigma^z_i sigma^z_j - Gamma sum_i sigma^x_i,
 * whose connected configurations are the N single spin flips (Sec. 2; all
 * off-diagonal elements -Gamma, so psi > 0 with zero phase).
 *   N        sites (2 <= N <= 512); bonds (p, p+1), and (N-1, 0) when periodic (N > 2)
 *   J, Gamma couplings (the paper's workload: open chain, J = Gamma = 1, N up to 384)
 *   other arguments as vqnqs_create, with n_max = N in the weight blob.
 * Every entry point except vqnqs_local_energy_ragged accepts such a context;
 * any configuration of N bits is a valid sample. */
int vqnqs_create_tfim(int N, int periodic, double J, double Gamma, int layers, int d_model, int heads, int K,
                      const float* weights, vqnqs_ctx** out);

/* Create an L x L Heisenberg context with the paper's architecture variants
 * (Sec. 3.1 and Table 1):
 *   vq_heads    the vector quantizers have vq_heads heads (Eq. vq with H
 *               heads; Table 1 uses H in {1, 2, 4, 8} with 64 codes each): the
 *               attention output o is split into vq_heads segments of
 *               d_model / vq_heads values, segment h goes to its nearest
 *               codeword among the K of its own codebook, and the quantized
 *               vector is the concatenation.  K is the codewords per head;
 *               vq_heads in 1..8, d_model / vq_heads a multiple of 8.  A row's
 *               code packs c_h in bits [h * b, (h + 1) * b), b = ceil(log2 K),
 *               32 / b heads per 32-bit word, at most two words (64 codes: up
 *               to 5 heads in one word, Table 1's 8 heads = 48 bits in two;
 *               two-word codes are given a dense id per chunk before the
 *               per-location deduplication, and vqnqs_codes /
 *               vqnqs_local_energy_codes refuse them).  Each layer's codebook
 *               block (K * d_model floats) is read as
 *               [vq_heads][K][d_model / vq_heads].
 *   token_group G in {1, 2, 4}: each token is a group of G consecutive spins
 *               (Sec. 3.1 tokens as particle groups): the token at position t
 *               is the value of group t - 1, sum_k s[(t-1) G + k] 2^k, with
 *               begin-of-sequence 2^G at t = 0; the blob holds 2^G + 1 token
 *               embeddings, N / G position embeddings and a 2^G-way head
 *               (W_head [d][2^G], b_head [2^G]); log psi = 1/2 sum_t log
 *               P(group t | earlier groups); rows per configuration are N / G
 *               and vqnqs_codes returns [B][layers][N / G].  N % G == 0.
 *   half_block  nonzero: Table 1's final half-block follows the blocks,
 *               x <- x + attention(LN(x)) W_o + b_o with its own LN, W_qkv and
 *               W_o and no quantizer or MLP; its weights (LN gain and shift,
 *               W_qkv [d][3d], b_qkv, W_o [d][d], b_o) sit between the last
 *               block and LN_f in the blob, which then has
 *               vqnqs_num_params_arch(L*L, layers, d_model, K, 1, G) values.  Its
 *               outputs are not quantized: the output projection and the head
 *               run per active row.
 * vq_heads = 1, half_block = 0, token_group = 1 is vqnqs_create.  With several heads the
 * quantizer search runs per head on the CUDA cores (FP32 distances, lowest
 * index on ties).  Local energies and log psi accept every flag combination;
 * VQNQS_INCREMENTAL with several heads needs a one-word code (heads x bits <= 32)
 * and K <= 1024, and certifies a row when ||delta|| is below the smallest
 * radius over its segments (each segment's code then provably stays);
 * the final half-block and G > 1 refuse it.  vqnqs_grad_log_psi, vqnqs_sample and
 * vqnqs_vmc_step return VQNQS_ERR_ARG for any variant, vqnqs_vq_assign for
 * several heads, vqnqs_local_energy_ragged for G > 1; vqnqs_codes returns
 * packed codes.  The FLOP counters of
 * vqnqs_get_stats cover the quantized blocks only. */
int vqnqs_create_arch(int L, int periodic, double J, int layers, int d_model, int heads, int K, int vq_heads,
                      int half_block, int token_group, const float* weights, vqnqs_ctx** out);

/* Weight blob size of a model with the final half-block (half_block != 0) or
 * without, and tokens of token_group spins (0 for an invalid group size). */
size_t vqnqs_num_params_arch(int n_max, int layers, int d_model, int K, int half_block, int token_group);

/* Replace the weights (HOST blob when is_device == 0, DEVICE blob otherwise) and
 * rebuild the derived tables on `stream`. */
int vqnqs_set_weights(vqnqs_ctx* ctx, const float* weights, int is_device, void* stream);

/* Workspace bytes for the calls below with `flags`, sized for chunks of up to
 * `chunk_samples` samples (<= 0 picks the library default).  A call given a
 * smaller workspace processes fewer samples per chunk; the minimum is one sample. */
size_t vqnqs_workspace_bytes(const vqnqs_ctx* ctx, int chunk_samples, int flags);

/* log psi(s) = 1/2 sum_p log P(s_p | s_<p) for B samples (Sec. 2 polar form, chain rule).
 *   dev_spins   DEVICE uint8 [B][N]
 *   dev_log_psi DEVICE float [B] (output)
 *   flags       VQNQS_REUSE | VQNQS_BF16
 *   dev_ws      DEVICE workspace of ws_bytes bytes, 256-byte aligned */
int vqnqs_log_psi(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, float* dev_log_psi, int flags,
                  void* dev_ws, size_t ws_bytes, void* stream);

/* Local energies (Sec. 2, Eq. local-energy; per-location reuse of Sec. 3.2)
 * of a ragged batch: n_groups (1..8) groups of samples of different lattice
 * sizes (Sec. 4 evaluates 4x4 to 12x12 lattices with one architecture)
 * evaluated with the context's model, all groups sharing one pipeline (chunks
 * mix lattice sizes; deduplication of per-location work spans the groups of a
 * chunk).
 *   L_g, B_g     HOST int [n_groups]: lattice side (2 .. L of the context) and sample
 *                count of each group; boundary conditions and J are the context's
 *   dev_spins    DEVICE uint8: the groups' samples concatenated, group after group,
 *                L_g^2 bytes per sample
 *   dev_e_loc    DEVICE float [sum B_g] (output), same order
 *   dev_mean_var DEVICE double [2] (output, may be NULL): FP64 mean and variance over all
 * Position embeddings are shared: site p of every lattice uses row p. */
int vqnqs_local_energy_ragged(vqnqs_ctx* ctx, int n_groups, const int* L_g, const int* B_g,
                              const uint8_t* dev_spins, float* dev_e_loc, double* dev_mean_var, int flags,
                              void* dev_ws, size_t ws_bytes, void* stream);

/* The codeword index chosen at every layer and position (Sec. 3.1, Eq. vq; the
 * indices the paper keeps "for bookkeeping") when log psi of B configurations
 * is evaluated as given (no connected configurations):
 *   dev_codes    DEVICE int32 [B][layers][N] (output)
 *   dev_log_psi  DEVICE float [B] (output, may be NULL when B <= 65536)
 * Same flags, workspace and stream rules as vqnqs_log_psi. */
int vqnqs_codes(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, int* dev_codes, float* dev_log_psi, int flags,
                void* dev_ws, size_t ws_bytes, void* stream);

/* Autoregressive direct sampling (Sec. 2: psi = sqrt(P) with P a product of
 * conditionals, so configurations are drawn exactly from |psi|^2 one site at a
 * time, without a Markov chain).  Site p of sample b is up when
 * dev_uniforms[b][p] < P(s_p = up | s_<p); the random numbers are the caller's.
 *   dev_uniforms DEVICE float [B][N], values in [0, 1)
 *   dev_spins    DEVICE uint8 [B][N] (output)
 *   dev_log_psi  DEVICE float [B] (output): log psi of the drawn configurations
 *   flags        VQNQS_BF16 for the tensor-core GEMMs (others ignored)
 *   dev_ws       DEVICE workspace (vqnqs_sample_workspace_bytes), 256-byte aligned;
 *                a smaller one draws fewer samples at a time (minimum one)
 * Each position runs every block on the batch's rows with the keys and values
 * of the earlier positions kept in the workspace. */
size_t vqnqs_sample_workspace_bytes(const vqnqs_ctx* ctx, int chunk_samples, int flags);
int vqnqs_sample(vqnqs_ctx* ctx, int B, const float* dev_uniforms, uint8_t* dev_spins, float* dev_log_psi,
                 int flags, void* dev_ws, size_t ws_bytes, void* stream);

/* One variational Monte Carlo step (Sec. 2): B configurations drawn from
 * |psi|^2 with the given uniforms (vqnqs_sample), their local energies, the
 * energy gradient grad_k = 2 mean[(E_loc - mean E_loc) O_k] (vqnqs_grad_log_psi,
 * Eq. st for the quantizers), then the weights updated in place,
 * theta <- theta - lr * grad (in FP32, the product and the difference each
 * rounded), and their derived tables rebuilt.
 *   dev_uniforms DEVICE float [B][N];  lr the step size
 *   dev_spins    DEVICE uint8 [B][N] (output: the drawn configurations)
 *   dev_e_loc    DEVICE float [B] (output)
 *   dev_grad     DEVICE float [P] (output: the gradient that was applied)
 *   dev_mean_var DEVICE double [2] (output: FP64 mean and variance of E_loc)
 *   flags        as vqnqs_local_energy (they also select the sampler's GEMMs)
 *   dev_ws       DEVICE workspace of vqnqs_vmc_workspace_bytes(ctx, B, flags) bytes */
size_t vqnqs_vmc_workspace_bytes(const vqnqs_ctx* ctx, int B, int flags);
int vqnqs_vmc_step(vqnqs_ctx* ctx, int B, const float* dev_uniforms, float lr, uint8_t* dev_spins, float* dev_e_loc,
                   float* dev_grad, double* dev_mean_var, int flags, void* dev_ws, size_t ws_bytes, void* stream);

/* Copies the context's current weight blob (vqnqs_num_params floats) to dev_weights. */
int vqnqs_get_weights(vqnqs_ctx* ctx, float* dev_weights, void* stream);

/* Local energies (Sec. 2, Eq. local-energy) of B samples.
 *   dev_e_loc     DEVICE float [B] (output): per-lattice E_loc(s) in units of J S.S
 *   dev_mean_var  DEVICE double [2] (output, may be NULL): FP64 mean and variance
 *                 (1/B normalisation) of the B local energies
 *   dev_log_psi   DEVICE float [B] (output, may be NULL): log psi of the samples
 * Every configuration one nearest-neighbour exchange away from a sample is
 * evaluated (Sec. 2: O(N) non-zero entries per row).
 *   flags         VQNQS_REUSE | VQNQS_BF16 | VQNQS_INCREMENTAL (the last needs the first) */
int vqnqs_local_energy(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, float* dev_e_loc,
                       double* dev_mean_var, float* dev_log_psi, int flags,
                       void* dev_ws, size_t ws_bytes, void* stream);

/* vqnqs_local_energy that also returns the codeword chosen (Sec. 3.1, Eq. vq)
 * at every layer and position of every configuration it evaluated: the
 * sample (configuration 0) and its connected configurations (1, 2, ... in
 * bond order: site p = y L + x contributes its bond to ((x+1) mod L, y), then
 * to (x, (y+1) mod L), wrapped bonds only when periodic; a bond enters when its
 * two spins differ), or the N single flips in site order for the Ising chain.
 *   dev_codes  DEVICE int32 [B][1 + max_conn][layers][N], max_conn = the number of
 *              bonds (sites for the chain); slots of configurations a sample does
 *              not have are left as they were
 * A row before its configuration's first changed position reports the sample's
 * code there (causality: the same inputs).  Same flags, workspace and stream
 * rules as vqnqs_local_energy; each layer adds one copy kernel. */
int vqnqs_local_energy_codes(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, float* dev_e_loc, int* dev_codes,
                             int flags, void* dev_ws, size_t ws_bytes, void* stream);

/* Gradient of log psi through the straight-through quantizer (Sec. 3.1,
 * Eq. st: the forward uses the nearest codeword, the backward flows through
 * softmax(-||o - W_j||)), and the VMC energy gradient (Sec. 2):
 *     O[b][k] = d log psi(s_b) / d theta_k        (theta in weight-blob order, P floats)
 *     grad[k] = sum_b w_b O[b][k]
 * with w_b = seeds[b] when dev_seeds is given, w_b = 2 (E_loc(s_b) - mean E_loc) / B
 * (the energy gradient 2 mean[(E_loc - mean E_loc) O_k]) when dev_e_loc is
 * given, else w_b = 1.
 *   dev_spins   DEVICE uint8 [B][N]
 *   dev_seeds   DEVICE float [B] or NULL;  dev_e_loc  DEVICE float [B] or NULL (not both)
 *   dev_O       DEVICE float [B][P] or NULL (per-sample gradients)
 *   dev_grad    DEVICE float [P] or NULL (at least one of O, grad)
 *   flags       VQNQS_BF16: the summed gradient's contractions (dX = dY W^T, dW = X^T dY
 *               and the recomputed forward GEMMs) run on the tensor cores with split
 *               operands (hi + lo BF16 pairs, three MMAs, FP32 accumulation) when
 *               d_model % 64 == 0, K % 64 == 0, the chunk's rows are a multiple of 8,
 *               one quantizer head, no half-block and single-spin tokens; the per-sample
 *               O path, the attention backward and the row-wise steps stay FP32
 * Activations are recomputed layer by layer from the stored residual stream.
 * Scratch: vqnqs_grad_workspace_bytes(ctx, B, chunk_samples) bytes. */
size_t vqnqs_grad_workspace_bytes(const vqnqs_ctx* ctx, int B, int chunk_samples);
int vqnqs_grad_log_psi(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, const float* dev_seeds,
                       const float* dev_e_loc, float* dev_O, float* dev_grad, int flags, void* dev_ws,
                       size_t ws_bytes, void* stream);

/* The energy gradient of samples sharded over ranks (one GPU each), with one
 * exchange step (Sec. 2 gradient estimator: grad_k = 2 mean[(E - mean E) O_k]).
 * Since sum_b (E_b - Ebar) O_b = sum_b E_b O_b - Ebar sum_b O_b, each rank sums
 * over its own samples
 *     partials[0 .. P)      sum_b E_b O_b[k]
 *     partials[P .. 2P)     sum_b O_b[k]
 *     partials[2P], [2P+1]  sum_b E_b, sum_b E_b^2
 *     partials[2P+2]        its sample count
 * (FP64, P = vqnqs_num_params floats of the blob), the ranks add these 2P + 3
 * values with one all-reduce (the caller's collective, e.g. NCCL), and
 * vqnqs_energy_grad_combine turns the sums into grad (FP32 [P]) and the FP64
 * mean and variance of E_loc over all ranks' samples.
 *   dev_e_loc   DEVICE float [B]: the rank's local energies
 *   dev_partials DEVICE double [2P + 3] (output; zeros when B = 0)
 *   dev_ws      DEVICE workspace of vqnqs_energy_grad_partials_workspace_bytes(ctx, B, chunk)
 * The two sums take two backward passes (vqnqs_grad_log_psi with seeds E and 1),
 * each summed in FP32.  Same model restrictions as vqnqs_grad_log_psi. */
size_t vqnqs_energy_grad_partials_workspace_bytes(const vqnqs_ctx* ctx, int B, int chunk_samples);
int vqnqs_energy_grad_partials(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, const float* dev_e_loc,
                               double* dev_partials, int flags, void* dev_ws, size_t ws_bytes, void* stream);
/*   dev_partials  DEVICE double [2P + 3]: the all-reduced partials (any number of ranks)
 *   dev_grad      DEVICE float [P] (output): 2 (sum E O - Ebar sum O) / n
 *   dev_mean_var  DEVICE double [2] (output, may be NULL): Ebar and sum E^2 / n - Ebar^2 */
int vqnqs_energy_grad_combine(vqnqs_ctx* ctx, const double* dev_partials, float* dev_grad, double* dev_mean_var,
                              void* stream);

/* The per-location tensor-core GEMM on its own (the kernel behind the QKV and
 * MLP steps of the BF16 path, Sec. 3.2 per-location operations):
 *     C[M][N] = A[M][K] @ Bt[N][K]^T + bias[N]   (+ epilogue)
 *   A, Bt      DEVICE bfloat16, row-major with K contiguous (Bt is the weight
 *              stored [out][in])
 *   bias       DEVICE float [N]
 *   epilogue   0: C bfloat16 [M][N];  1: C bfloat16 of GELU(.);
 *              2: C float [M][N] = . + R[M][N] (R DEVICE float);  3: C float;
 *              4: C float of GELU(.).  GELU(x) = x (1 + erf(x / sqrt 2)) / 2 with
 *              erf by Abramowitz & Stegun 7.1.26 (absolute error <= 1.5e-7 plus
 *              FP32 rounding).  Output chunks of 32 full rows leave through TMA
 *              stores, the others row by row; C rows at or past M are not written.
 * Needs K % 64 == 0, N % 64 == 0 and 16-byte aligned pointers (else
 * VQNQS_ERR_ARG).  BF16 x BF16 products, FP32 accumulation; asynchronous on
 * `stream`; a stalled pipeline sets VQNQS_DEV_TIMEOUT in the status word. */
int vqnqs_gemm_bf16(vqnqs_ctx* ctx, int M, int N, int K, const void* dev_A, const void* dev_Bt,
                    const float* dev_bias, const float* dev_R, void* dev_C, int epilogue, void* stream);

/* vqnqs_gemm_bf16 with split operands (the GEMMs of VQNQS_BF16_SPLIT, Sec. 3.2
 * per-location operations in FP32-grade arithmetic on the BF16 tensor cores):
 *   A2   DEVICE bfloat16 [2M][K]: rows 0..M-1 hold hi = bf16(a), rows M..2M-1 lo = bf16(a - hi)
 *   Bt2  DEVICE bfloat16 [2N][K]: the same for the weight stored [out][in]
 *   C    epilogues 0, 1: bfloat16 [2M][N], hi rows then lo rows of the result;
 *        epilogues 2, 3, 4: float [M][N] as in vqnqs_gemm_bf16
 * C = A_hi Bt_hi^T + A_hi Bt_lo^T + A_lo Bt_hi^T + bias (+ epilogue), three BF16
 * MMA passes into one FP32 accumulator.  Same limits and errors as vqnqs_gemm_bf16,
 * and M <= 2^29. */
int vqnqs_gemm_bf16_split(vqnqs_ctx* ctx, int M, int N, int K, const void* dev_A2, const void* dev_Bt2,
                          const float* dev_bias, const float* dev_R, void* dev_C, int epilogue, void* stream);

/* Nearest codeword of R vectors under layer `layer`'s codebook (Sec. 3.1, Eq. vq):
 * code[r] = argmin_j ||W_j||^2 - 2 O[r] . W_j, lowest j on exact ties.
 *   dev_O     DEVICE float [R][d_model] (16-byte aligned);  dev_code  DEVICE int32 [R] (output)
 *   use_tensor_cores  0: FP32 FFMA kernel;  1: tensor-core kernel with split-TF32
 *             products (FP32-grade; needs K % 16 == 0, K <= 512, d_model % 32 == 0)
 * R is limited to 2^22 per call.  Near ties (relative gap < 1e-6) are counted
 * in the statistics.  Asynchronous on `stream`. */
int vqnqs_vq_assign(vqnqs_ctx* ctx, int layer, int R, const float* dev_O, int* dev_code, int use_tensor_cores,
                    void* stream);

/* The compressed (I, V) representation of Sec. 3.2 as a standalone step: every
 * distinct (row id, code) pair among R rows gets a dense new id.
 *   dev_uid, dev_code   DEVICE int32 [R]; 0 <= uid < 2^31, 0 <= code < 65536
 *   dev_new_id          DEVICE int32 [R] (output): new id of each row
 *   dev_rep_uid, dev_rep_code  DEVICE int32 [R] (output): the pair of each new
 *                       id, in entries 0 .. U-1
 *   dev_count           DEVICE int32 [1] (output): U, the number of distinct pairs
 *   dev_ws, ws_bytes    DEVICE scratch (256-byte aligned) of at least
 *                       vqnqs_compress_workspace_bytes(R) bytes for the hash table
 * New ids are dense in [0, U); which pair gets which id is unspecified.
 * Asynchronous on `stream`; probe-bound overruns set VQNQS_DEV_HASH_OVERFLOW. */
size_t vqnqs_compress_workspace_bytes(int R);
int vqnqs_compress_rows(vqnqs_ctx* ctx, int R, const int* dev_uid, const int* dev_code, int* dev_new_id,
                        int* dev_rep_uid, int* dev_rep_code, int* dev_count, void* dev_ws, size_t ws_bytes,
                        void* stream);

/* vqnqs_compress_rows for callers that cannot allocate device memory (for
 * example code running while a stream is captured into a CUDA graph, or a
 * host application that owns all device memory): same inputs, outputs and
 * result as vqnqs_compress_rows, but no context and no workspace.  Its hash
 * table is a file-scope device array of 6 MiB that every GPU loading the
 * library keeps until exit.  (Not a step of the paper; it has no counterpart
 * there.)
 *   R  0 .. VQNQS_NOALLOC_MAX_ROWS, else VQNQS_ERR_ARG
 * Allocates nothing (no cudaMalloc, no allocating library call).  The first
 * call on a device looks up the array's address with cudaGetSymbolAddress
 * (VQNQS_ERR_CUDA if that fails): make it before any stream capture.  All
 * calls on a device share the array; each call clears what it uses first, but
 * calls whose kernels overlap on the GPU race and give wrong results.  A
 * probe-bound overrun (which a table of twice the rows does not reach) sets
 * *dev_count to -1 instead of U.  After cudaDeviceReset the cached address is
 * stale: do not call this again in that process.
 * Asynchronous on `stream`. */
#define VQNQS_NOALLOC_MAX_ROWS (1 << 18)
int vqnqs_compress_rows_noalloc(int R, const int* dev_uid, const int* dev_code, int* dev_new_id,
                                int* dev_rep_uid, int* dev_rep_code, int* dev_count, void* stream);

/* Autotuner of the per-location tensor-core GEMMs: for each of the QKV, MLP up and
 * MLP down steps it times every output tile width (64, 128, 192, 256 columns)
 * that divides the step's output width on M rows (M >= 128, e.g. the typical
 * number of unique rows of a chunk), keeps the fastest for this context and
 * reports the average milliseconds per launch (-1 for widths that do not apply).
 * Synchronises `stream`.  Scratch: M * d_model * 40 bytes of workspace.
 * Needs d_model % 64 == 0. */
typedef struct vqnqs_tuning {
    int qkv_bn, mlp_up_bn, mlp_down_bn;
    float ms[3][4];  /* [step][width 64, 128, 192, 256] */
} vqnqs_tuning;
int vqnqs_autotune(vqnqs_ctx* ctx, int M, void* dev_ws, size_t ws_bytes, vqnqs_tuning* out, void* stream);

/* Chunk-size tuner of the local-energy path: for each candidate chunk size
 * (samples per chunk, HOST int cand[n_cand]) whose workspace fits ws_bytes,
 * evaluates the local energies of the B DEVICE samples once untimed and twice
 * timed with `flags`, writes the average milliseconds per evaluation to HOST
 * ms[i] (-1 when the candidate does not fit) and the fastest candidate to
 * *best.  Larger chunks mean fewer, larger launches; the caller then sizes its
 * workspace with vqnqs_workspace_bytes(ctx, *best, flags).  B <= 65536;
 * synchronises `stream`. */
int vqnqs_autotune_chunk(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, int flags, const int* cand, int n_cand,
                         void* dev_ws, size_t ws_bytes, int* best, float* ms, void* stream);

/* Work-split tuner of the incremental path's tensor-core kernels (BF16 flags with
 * VQNQS_INCREMENTAL; the workspace as for vqnqs_local_energy with these flags):
 * times the local energies of the B DEVICE samples (once untimed, twice timed per
 * setting) for the patch kernel's work items per CTA in {2, 4, 8}, keeps the
 * fastest, then for the changed-row kernel's items per SM in {1, 2, 4, 8, 16}, and keeps
 * both for this context (defaults 4 and 2).  Results do not depend on the setting
 * (each row is computed from its own inputs); only the assignment of work to CTAs
 * changes.  Writes the average milliseconds per evaluation to out (-1: not run).
 * B <= 65536; synchronises `stream`. */
typedef struct vqnqs_inc_tuning {
    int patch_items, rows_slices;
    float patch_ms[3];  /* items per CTA 2, 4, 8 */
    float rows_ms[5];   /* items per SM 1, 2, 4, 8, 16 */
} vqnqs_inc_tuning;
int vqnqs_autotune_incremental(vqnqs_ctx* ctx, int B, const uint8_t* dev_spins, int flags, void* dev_ws,
                               size_t ws_bytes, vqnqs_inc_tuning* out, void* stream);

/* Snapshot of the counters; synchronises the device first. */
int vqnqs_get_stats(vqnqs_ctx* ctx, vqnqs_stats* out);

/* Failure-path check: launches a kernel whose bounded wait on an mbarrier that
 * nothing arrives on gives up after about limit_cycles SM cycles (1 .. 4e9) and
 * sets VQNQS_DEV_TIMEOUT in the device status word, the same path every
 * tensor-core kernel takes when a pipeline stalls.  The context stays usable.
 * Asynchronous on `stream`; read the bit with vqnqs_get_stats. */
int vqnqs_check_timeout_path(vqnqs_ctx* ctx, long long limit_cycles, void* stream);

/* Zero the counters and the device status word. */
int vqnqs_reset_stats(vqnqs_ctx* ctx);

/* Per-stage timing.  While enabled, every stage of the path is bracketed by
 * CUDA events recorded on the stream it is launched on; vqnqs_profile_read
 * synchronises the device and returns, per stage, the number of kernel
 * launches and the summed event time since the last read (then clears them).
 * Stage names: config, active_rows, embed, ln1, qkv_gemm, attention, vq_argmin, dedupe,
 * post_ln, mlp_up, mlp_down, head, eloc, mean_var, backward, inc_certificate,
 * inc_classify, inc_patch, inc_recompute, inc_recompute_whole, half_block,
 * inc_exact_delta, bwd_recompute, bwd_gemm, bwd_attention, bwd_rowwise (the last
 * four inside backward). */
typedef struct vqnqs_stage_time {
    char name[24];
    int64_t calls;     /* times the stage ran */
    int64_t launches;  /* kernel launches it issued */
    double ms;         /* summed CUDA-event time */
} vqnqs_stage_time;

#define VQNQS_MAX_STAGES 32

int vqnqs_profile_enable(vqnqs_ctx* ctx, int enable);

/* Fills out[0 .. *n_out-1] (at most max_stages entries). */
int vqnqs_profile_read(vqnqs_ctx* ctx, vqnqs_stage_time* out, int max_stages, int* n_out);

/* Kernel launches issued by this context since it was created (host counter). */
int64_t vqnqs_launch_count(const vqnqs_ctx* ctx);

/* Last error message of this context ("" if none); valid until the next call. */
const char* vqnqs_last_error(const vqnqs_ctx* ctx);

/* Free the context and everything it owns.  NULL is ignored. */
void vqnqs_destroy(vqnqs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VQNQS_H */
