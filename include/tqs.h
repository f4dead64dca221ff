/*
 * tqs.h -- C ABI of the GB300 (sm_103a) noisy Monte-Carlo state-vector simulator
 * with tree-based reuse of intermediate states (TQSim, arXiv 2203.13892).
 *
 * The problem statement these calls follow (Sec. 2.4, 3.1, 3.2):
 *   a circuit (ordered gate list on n qubits) is run for N noisy shots; after every
 *   gate a depolarizing noise site may insert a random Pauli on that gate's
 *   qubits; each shot ends in a measurement whose bits may flip (readout error).
 *   The baseline simulator runs every shot from |0...0>.  Tree mode partitions the
 *   circuit into k+1 subcircuits with arities (A_0..A_k): instance m of level i
 *   starts from the stored state of its parent m / A_i, so intermediate states are
 *   reused by A_i children (Sec. 3.1, Eq. circuit-instances read as
 *   M_i = prod_{j<=i} A_j); the leaves are the N measured outcomes.
 *
 * Conventions
 *   - qubit q is bit q of the amplitude index and of the histogram bin;
 *   - two-qubit matrices act on the local index k = bit(q0) + 2*bit(q1);
 *     for CX, q0 is the control;
 *   - the noise site after gate g is numbered g (0-based, gate order); its
 *     Pauli is drawn with Philox4x32-10 keyed by the seed and the counter
 *     (node_lo, node_hi, g, 1); an error occurs iff word0 < floor(p*2^32); the
 *     Pauli index is 1 + (word1 * npaulis) >> 32 with npaulis = 3 (X,Y,Z) for
 *     one-qubit and 15 for two-qubit gates (index t -> P_{t>>2} on q0 and
 *     P_{t&3} on q1, with I,X,Y,Z = 0..3);
 *   - leaf m is measured with u = ((w0>>5)*2^26 + (w1>>6)) * 2^-53 drawn from
 *     counter (m_lo, m_hi, 0, 2): the outcome is the smallest y whose running sum
 *     of |psi_y|^2 exceeds u * sum|psi|^2; bit q then flips iff the word0 of
 *     counter (m_lo, m_hi, q, 3) is below floor(pm*2^32).
 *
 * Errors: every call returns a tqs_status and leaves its outputs untouched on
 * error; tqs_last_error() gives a thread-local message for the last failure.
 * Handles are owned by the library until their destroy call; every buffer
 * passed in is owned by the caller.  Device-side failures are reported as
 * TQS_ECUDA (or TQS_ETIMEOUT for a bounded wait that gave up); no kernel traps.
 */
#ifndef TQS_PUBLIC_API_H_
#define TQS_PUBLIC_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TQS_ABI_VERSION 1
#define TQS_MAX_LEVELS 17
#define TQS_MAX_QUBITS 30

typedef enum {
    TQS_OK = 0,
    TQS_EINVAL = 1,       /* malformed argument (qubit out of range, p outside [0,1], ...) */
    TQS_ENOMEM = 2,       /* host or device allocation failed / workspace too small */
    TQS_ECUDA = 3,        /* a CUDA call failed (message in tqs_last_error) */
    TQS_ETIMEOUT = 4,     /* a bounded device wait gave up */
    TQS_EUNSUPPORTED = 5, /* valid request outside what this library supports */
    TQS_EBOUNDS = 6       /* a device-side index check (TQS_FLAG_DEBUG_BOUNDS) found an index out of
                             range; the offending access was skipped and the results are invalid */
} tqs_status;

typedef enum {
    TQS_H = 0, TQS_X, TQS_Y, TQS_Z, TQS_S, TQS_SDG, TQS_T, TQS_TDG,
    TQS_RX, TQS_RY, TQS_RZ, TQS_P,
    TQS_CX, TQS_CZ, TQS_CP, TQS_SWAP,
    TQS_U1, /* arbitrary 2x2 matrix in `mat` */
    TQS_U2  /* arbitrary 4x4 matrix in `mat` */
} tqs_gate_kind;

/* One gate.  theta is used by RX/RY/RZ/P/CP; mat (interleaved re,im, row-major,
 * 2x2 for U1 and 4x4 for U2) is read only for U1/U2 and may be NULL otherwise.
 * q1 is ignored for one-qubit gates.  The matrix is copied at creation. */
typedef struct {
    uint32_t kind, q0, q1;
    double theta;
    const double *mat;
} tqs_gate;

typedef struct tqs_circuit tqs_circuit; /* opaque, library-owned */
typedef struct tqs_noise tqs_noise;     /* opaque, library-owned */
typedef struct tqs_plan tqs_plan;       /* opaque, library-owned */

/* Circuit from an ordered gate list (Sec. 2.2).  n_qubits in [1, TQS_MAX_QUBITS];
 * n_gates may be 0.  EINVAL on an unknown kind, a qubit >= n_qubits, q0 == q1
 * for a two-qubit gate, a non-finite angle or a NULL matrix for U1/U2. */
tqs_status tqs_circuit_create(uint32_t n_qubits, const tqs_gate *gates, size_t n_gates,
                              tqs_circuit **out);
void tqs_circuit_destroy(tqs_circuit *c);

/* Noise model (Sec. 4.3): depolarizing probability p1 after one-qubit gates, p2
 * after two-qubit gates (probability of a non-identity Pauli, uniform over the
 * 3 or 15 choices), readout bit-flip probability pm.  Each in [0,1] else EINVAL. */
tqs_status tqs_noise_model(double p1, double p2, double pm, tqs_noise **out);
void tqs_noise_destroy(tqs_noise *nz);

/* Noise model with the non-unitary channels of Sec. 4.3 as well.  After every
 * gate and its depolarizing Pauli, each of the gate's qubits (q0, then q1) goes
 * through, in this order: thermal relaxation (when t1 > 0: amplitude damping
 * with gamma = 1 - exp(-t/T1) then phase damping with
 * lambda = 1 - exp(t/T1 - 2t/T2), t = time_1q or time_2q by the gate's arity;
 * needs 0 < T2 <= 2 T1), amplitude damping with ad_gamma, phase damping with
 * pd_lambda.  Each channel is one quantum-trajectory step: with P1 the
 * probability of the qubit being 1 in the normalised state, the jump operator
 * (amplitude damping sqrt(gamma)|0><1|, phase damping sqrt(lambda)|1><1|) is
 * chosen with probability rate * P1, else diag(1, sqrt(1 - rate)), and the
 * state is renormalised; the choice compares u = ((w0>>5)*2^26 + (w1>>6)) * 2^-53
 * of Philox4x32-10 counter (node_lo, node_hi, 16 g + 8 i + c, 4) with rate * P1
 * (g the gate, i = 0/1 its qubit, c = 0..3 the channel in the order above).
 * Rates and probabilities in [0, 1], times >= 0, else EINVAL.  A zero rate
 * (t1 = 0) means no such channel.  Every gate with a channel ends a tile pass:
 * the channel's choice needs a reduction over the whole state. */
typedef struct {
    double p1, p2, pm;
    double ad_gamma, pd_lambda;
    double t1, t2, time_1q, time_2q;
} tqs_noise_params;
tqs_status tqs_noise_model_ex(const tqs_noise_params *params, tqs_noise **out);

typedef enum { TQS_MODE_BASELINE = 0, TQS_MODE_TREE = 1 } tqs_mode;
typedef enum { TQS_FP64 = 0, TQS_FP32 = 1 } tqs_precision;
typedef enum {
    TQS_PART_DCP = 0,      /* dynamic circuit partition (Sec. 3.2) */
    TQS_PART_UCP = 1,      /* uniform: k+1 levels of equal arity (Sec. 3.2.1) */
    TQS_PART_XCP = 2,      /* exponential: A_i = a * 2^(k-i) (Sec. 3.2.1) */
    TQS_PART_EXPLICIT = 3, /* caller's arity[] and split[] */
    TQS_PART_LEARNED = 4   /* learned partitioner (tqs_learned_set_model), DCP as fallback */
} tqs_partitioner;

#define TQS_FLAG_NO_FIDELITY 0x1u /* skip the ideal run and the fidelity (fidelity = NaN) */
#define TQS_FLAG_PROFILE 0x2u     /* time every launch with CUDA events (report.prof_*) */
#define TQS_FLAG_AUTOTUNE 0x4u    /* choose tile_qubits (and, for FP32, fusion) by timing trial runs,
                                     cached per circuit shape */
#define TQS_FLAG_FUSE 0x8u        /* FP32, tiles of 2^11 / 2^12: apply each block of >= 2 consecutive dense
                                     gates on t - 7 tile qubits as one fused 3xTF32 product on the tensor
                                     cores (off by default: on circuits whose blocks hold only a few gates
                                     the per-gate path is faster) */
#define TQS_FLAG_HOST_POOL 0x10u  /* keep every level's state slots in pinned host memory mapped into the
                                     device's address space, read and written in place by the kernels
                                     (Sec. 3.3-3.4: idle host memory holds the intermediate states; on a
                                     Grace-Blackwell node the accesses go over NVLink-C2C).  Without this
                                     flag, a plan whose library-allocated workspace cannot hold one node
                                     per level moves the upper levels' slots there by itself.  At most a
                                     quarter of the host's physical memory is pinned (the node batch
                                     shrinks to fit); ignored by tqs_simulate_static. */

#define TQS_FLAG_DEBUG_BOUNDS 0x20u /* every state-pass CTA checks, before its first memory access, that its
                                       output slot, input slot and every tile and outside-tile bit lie inside
                                       the buffers and the state; a CTA that fails writes the device error
                                       word, touches no memory and returns, and the call returns
                                       TQS_EBOUNDS (no trap).  Off by default: the check costs a few
                                       instructions per CTA. */
#define TQS_FLAG_FAULT_TIMEOUT 0x40u /* test only: fused tensor-core blocks (TQS_FLAG_FUSE) issue no MMA
                                        and no commit and wait with a short iteration cap, so their
                                        bounded wait gives up with no work in flight; the call returns
                                        TQS_ETIMEOUT and the library stays usable */
#define TQS_FLAG_FAULT_BOUNDS 0x80u  /* test only, with TQS_FLAG_DEBUG_BOUNDS: the executor tells the
                                        kernels that the output pool holds one slot fewer than it does,
                                        so the last node of a full launch fails the check above (no
                                        access is made out of range) */
#define TQS_FLAG_SPECIALIZE 0x100u  /* FP32 plans: compile, when the plan is created, one pass kernel per
                                       pass program (NVRTC, sm_103a): the pass's records become
                                       straight-line code with its tile layout as constants, in place
                                       of the generic kernel that interprets them.  Same arithmetic,
                                       fewer instructions; a few seconds of compilation per new
                                       circuit (kept for the life of the process, keyed by the
                                       program).  Passes with fused tensor-core blocks keep the
                                       generic kernel; FP64 plans ignore the flag.  Needs NVRTC
                                       (libnvrtc.so.13) and the driver at run time, else
                                       TQS_EUNSUPPORTED; refused by tqs_simulate_static, which must
                                       not allocate. */

/* Kernel classes timed under TQS_FLAG_PROFILE (index into report.prof_*). */
#define TQS_PROF_NOISE 0   /* Philox noise draws + Pauli frames */
#define TQS_PROF_STORE 1   /* tile pass that stores the node state */
#define TQS_PROF_SUMS 2    /* leaf tile pass that writes measurement block sums */
#define TQS_PROF_SAMPLE 3  /* per-leaf outcome pick + tile recompute */
#define TQS_PROF_KINDS 4

/* Options.  A zeroed struct is NOT the default: call tqs_options_default().
 *   z, eps       DCP confidence z and margin eps (defaults 1.96, 0.05)
 *   copy_gates   DCP minimum subcircuit length c in gates (default 10, Sec. 3.6)
 *   k            number of levels - 1 for UCP/XCP/EXPLICIT (levels = k+1 <= 17)
 *   arity, split EXPLICIT tree: arity[0..k], split[0..k+1] with split[0] = 0,
 *                split[k+1] = n_gates, non-decreasing; prod(arity) >= shots
 *   tile_qubits  maximum shared-memory tile width t in [6, 13] (0 = default: 12 FP32, 11 FP64)
 *   batch        node instances per launch (0 = chosen from the memory budget)
 *   workspace, workspace_bytes   optional caller-owned DEVICE buffer (>= 256-byte
 *                aligned) used for all scratch; NULL = the library allocates, at
 *                most workspace_bytes when that is nonzero
 *   stream       cudaStream_t to run on (NULL = legacy default stream)
 *   flags        TQS_FLAG_* bits */
typedef struct {
    tqs_mode mode;
    tqs_precision prec;
    tqs_partitioner part;
    double z, eps;
    uint32_t copy_gates;
    uint32_t k;
    const uint64_t *arity;
    const uint32_t *split;
    uint32_t tile_qubits;
    uint32_t batch;
    void *workspace;
    size_t workspace_bytes;
    void *stream;
    uint32_t flags;
} tqs_options;

void tqs_options_default(tqs_options *o);

/* Filled by tqs_simulate / tqs_plan_execute when non-NULL. */
typedef struct {
    uint64_t shots_done;
    uint32_t levels;                      /* k + 1 */
    uint64_t arity[TQS_MAX_LEVELS];
    uint32_t split[TQS_MAX_LEVELS + 1];
    uint64_t node_instances[TQS_MAX_LEVELS]; /* nodes simulated per level */
    uint32_t passes[TQS_MAX_LEVELS];         /* state passes per node per level */
    uint64_t kernel_launches;
    double kernel_ms;         /* device time of the simulation (CUDA events) */
    double shots_per_s;       /* shots_done / kernel_ms */
    double alg_bytes;         /* algorithmic state bytes moved (2 per stored node, 1 per leaf) */
    double fid_norm, fid_s;   /* normalized fidelity F and F_s vs the ideal run (NaN if skipped/undefined) */
    double theo_speedup;      /* levels * N / sum_i node_instances[i] */
    /* per kernel class (TQS_PROF_*), filled under TQS_FLAG_PROFILE: launches,
     * summed event time and algorithmic bytes (state reads + writes; a state is
     * 2^n amplitudes of 8 (FP32) or 16 (FP64) bytes) */
    uint64_t prof_launches[TQS_PROF_KINDS];
    double prof_ms[TQS_PROF_KINDS];
    double prof_bytes[TQS_PROF_KINDS];
    /* gate blocks per node per level applied as one fused 2^k x 2^k product on
     * the tensor cores (FP32 only; 0 when the per-gate path is used) */
    uint32_t fused_blocks[TQS_MAX_LEVELS];
} tqs_report;

/* Partition only (host, no GPU): the tree the options select for `shots`.
 * arity_out[TQS_MAX_LEVELS], split_out[TQS_MAX_LEVELS+1]; *levels_out = k+1. */
tqs_status tqs_partition(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                         const tqs_options *opts, uint32_t *levels_out, uint64_t *arity_out,
                         uint32_t *split_out);

/* Full simulation: plan, upload, run on the GPU, copy the histogram back.
 * counts: caller-owned HOST array of 2^n uint64 (overwritten; sums to shots).
 * fidelity: normalized fidelity F vs the noiseless run (NaN with TQS_OK when the
 * ideal distribution is uniform, or when TQS_FLAG_NO_FIDELITY is set). */
tqs_status tqs_simulate(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, uint64_t seed,
                        const tqs_options *opts, uint64_t *counts, double *fidelity,
                        tqs_report *report);

/* Device-resident execution (what a benchmark times): tqs_plan_create does the
 * host planning and uploads gate tables and workspace; tqs_plan_execute runs one
 * simulation with `seed`, accumulating into the caller's DEVICE array d_counts
 * (2^n uint64, zeroed by the call) on opts->stream, and returns without
 * synchronising (report fields needing the device are filled only when
 * `report` is non-NULL, which synchronises). */
tqs_status tqs_plan_create(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                           const tqs_options *opts, tqs_plan **out);
tqs_status tqs_plan_execute(tqs_plan *p, uint64_t seed, uint64_t *d_counts, tqs_report *report);
size_t tqs_plan_workspace_bytes(const tqs_plan *p);
/* Bytes of the plan's state pool held in mapped host memory (0 when all of it
 * is in device memory; see TQS_FLAG_HOST_POOL). */
size_t tqs_plan_host_pool_bytes(const tqs_plan *p);
void tqs_plan_destroy(tqs_plan *p);

/* Batched execution (many independent simulations, uneven sizes).  All
 * circuits are planned with the shared options (not EXPLICIT; workspace must be
 * NULL: the batch shares out device memory in proportion to 2^n), then their
 * launches are captured once into a CUDA graph with one branch per circuit.
 * tqs_batch_execute writes seeds[i] to device memory and replays the graph on the
 * batch's own stream (it returns after the replay finished); histogram i is then
 * read with tqs_batch_counts (HOST copy) or tqs_batch_device_counts (device
 * pointer, valid until the next execute or destroy).  The report, when given,
 * aggregates all circuits. */
typedef struct tqs_batch tqs_batch;
tqs_status tqs_batch_create(size_t count, const tqs_circuit *const *circuits, const tqs_noise *const *noises,
                            const uint64_t *shots, const tqs_options *opts, tqs_batch **out);
tqs_status tqs_batch_execute(tqs_batch *b, const uint64_t *seeds, tqs_report *report);
tqs_status tqs_batch_counts(const tqs_batch *b, size_t i, uint64_t *counts);
const uint64_t *tqs_batch_device_counts(const tqs_batch *b, size_t i);
size_t tqs_batch_size(const tqs_batch *b);
void tqs_batch_destroy(tqs_batch *b);

/* Learned partitioner (an addition to the paper, which has DCP only).  A small
 * network (TQS_LEARNED_FEATURES -> 128 -> 128 -> TQS_LEARNED_CLASSES, ReLU,
 * softmax, FP32, trained and run on the GPU by the library's own kernels)
 * chooses between candidate trees; class = 10*mode + k means k extra levels with
 * DCP's first-level sample-size rule (Sec. 3.2, Eq. sample_size_formula) and
 * equal lower arities, cut into equal parts (mode 0) or with every cut moved to
 * the nearest tile-pass boundary (mode 1).  DCP is the fallback and the arbiter: a
 * class is allowed only when its first-level arity A_0 is at least DCP's (no
 * wider Hoeffding bound on A_0) and it has no more levels than DCP; with no model
 * loaded, TQS_PART_LEARNED returns TQS_EUNSUPPORTED.
 * Parameters: one float array of tqs_learned_param_count() values, laid out
 * W1[F][128], b1[128], W2[128][128], b2[128], W3[128][C], b3[C]. */
#define TQS_LEARNED_FEATURES 40
#define TQS_LEARNED_CLASSES 20
size_t tqs_learned_param_count(void);
/* Host only: features (HOST float[TQS_LEARNED_FEATURES]) and, when non-NULL,
 * allowed[TQS_LEARNED_CLASSES] (1 = valid and judged acceptable against DCP). */
tqs_status tqs_learned_features(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                float *features, uint8_t *allowed);
/* Host only: the tree of candidate class `cls` (EINVAL if that class is invalid here). */
tqs_status tqs_learned_candidate(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                 uint32_t cls, uint32_t *levels_out, uint64_t *arity_out, uint32_t *split_out);
/* Training with Adam on the GPU: X HOST [rows][F], labels HOST [rows] in
 * [0, C); mini-batches of `batch` rows, `epochs` passes, learning rate lr;
 * init = NULL for a seeded He initialisation.  weights: HOST output. */
tqs_status tqs_learned_train(const float *X, const int32_t *labels, size_t rows, uint32_t epochs, uint32_t batch,
                             float lr, uint64_t seed, const float *init, float *weights, float *final_loss);
/* One forward + backward on the GPU: mean cross-entropy and its gradient (HOST
 * arrays; grad has tqs_learned_param_count() floats). */
tqs_status tqs_learned_loss_grad(const float *weights, const float *X, const int32_t *labels, size_t rows,
                                 float *loss, float *grad);
/* Forward on the GPU: logits HOST [rows][C]. */
tqs_status tqs_learned_predict(const float *weights, const float *X, size_t rows, float *logits);
/* Process-wide model used by TQS_PART_LEARNED (copied); NULL unloads it. */
tqs_status tqs_learned_set_model(const float *weights);

/* Debug / parity entry points.
 * tqs_debug_node_state: the logical state (2^n complex, interleaved FP64, HOST
 * array) of instance `node` of tree level `level` after its subcircuit, in the
 * tree the options select, including the global phase of the inserted Paulis.
 * tqs_debug_node_noise: the Pauli index (0 = none) drawn at each site of that
 * node's subcircuit (HOST array of split[level+1]-split[level] bytes). */
tqs_status tqs_debug_node_state(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                uint64_t seed, const tqs_options *opts, uint32_t level,
                                uint64_t node, double *psi_out);
tqs_status tqs_debug_node_noise(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                uint64_t seed, const tqs_options *opts, uint32_t level,
                                uint64_t node, uint8_t *paulis_out);
/* tqs_debug_plan_order (host only, no device call): the order in which the plan
 * applies the circuit's gates.  order_out[i] (HOST, n_gates entries) = the gate
 * index applied i-th (levels in turn, each level's passes in turn, each pass in
 * its program order); pass_out[i] = the global pass that applies it; tile_out
 * (optional, one entry per pass) = the pass's tile as a mask of physical qubits
 * (SWAPs are a relabelling: physical = where a logical qubit lives at that
 * point); *npasses_out = the number of passes.  Gates that share a physical
 * qubit appear in circuit order. */
tqs_status tqs_debug_plan_order(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                const tqs_options *opts, uint32_t *order_out, uint32_t *pass_out,
                                uint32_t *tile_out, uint32_t *npasses_out);
/* tqs_debug_spec_check (host only, no device call): builds the plan the options
 * select (FP32), generates the source of every kernel TQS_FLAG_SPECIALIZE would
 * compile for it and compiles each with NVRTC for sm_103a without loading it.
 * *nkernels_out = the kernels generated (passes with fused tensor-core blocks
 * have none); *src_bytes_out (optional) = their total generated source.  Returns
 * TQS_EUNSUPPORTED without NVRTC, TQS_EINVAL for FP64 options, TQS_ECUDA with
 * the compiler's log (tqs_last_error) if a kernel does not compile. */
tqs_status tqs_debug_spec_check(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                const tqs_options *opts, uint32_t *nkernels_out, uint64_t *src_bytes_out);
/* tqs_debug_spec_source (host only): the generated source of global pass `pass`
 * in mode `mode` (0 store, 1 sums, 2 sample): the tile-layout constants, then
 * the pass's records as statements, NUL-terminated in the HOST buffer `buf` of
 * `cap` bytes (truncated to fit); *len_out = the full length.  TQS_EINVAL for
 * a pass index out of range or FP64 options, TQS_EUNSUPPORTED when the pass has
 * no specialised form (fused tensor-core blocks). */
tqs_status tqs_debug_spec_source(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                 const tqs_options *opts, uint32_t pass, int mode, char *buf, uint64_t cap,
                                 uint64_t *len_out);

/* Simulation without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory, such as
 * code that runs while another component owns the whole device through its own
 * pool allocator, latency-critical loops where cudaMalloc/cudaFree would
 * synchronise the device, and plugin hosts that forbid allocation.
 *
 * It runs the same simulation as tqs_plan_create + tqs_plan_execute, but all
 * device scratch (gate tables, noise tables, Pauli frames, the state pool and
 * the measurement block sums) lives in one static array of
 * TQS_STATIC_SCRATCH_BYTES bytes inside the library, which every GPU that loads
 * the library keeps reserved until the process exits.  The node batch shrinks to
 * fit the array; a request that does not fit with one node per level returns
 * TQS_EINVAL and says how many bytes it needs.  opts->workspace, workspace_bytes
 * and TQS_FLAG_PROFILE are ignored.
 *
 * d_counts: caller-owned DEVICE array of 2^n uint64, zeroed by the call, then
 * the histogram (sums to shots).  The call runs on opts->stream and returns
 * after the simulation has finished; it uploads the plan's tables and
 * synchronises that stream, so it must not be called on a stream that is being
 * captured.  The first call on each device (with that device current) looks up
 * the array's device address and keeps it for the rest of the process; do not
 * call this again on a device after cudaDeviceReset() of that device.  Every
 * call shares the one array and it keeps the last call's contents: calls whose
 * GPU work overlaps (different streams or threads) race on it, so serialise
 * them.  opts->part = TQS_PART_LEARNED returns TQS_EUNSUPPORTED (the network
 * behind it allocates device memory). */
#define TQS_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
tqs_status tqs_simulate_static(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, uint64_t seed,
                               const tqs_options *opts, uint64_t *d_counts);

const char *tqs_last_error(void);
int tqs_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TQS_PUBLIC_API_H_ */
