// internal.h -- structures shared by the host planner, the executor and the CUDA
// kernels of libtqs (not part of the public ABI; see include/tqs.h).
#pragma once

// The device-visible part (constants and record layouts) is also compiled at
// run time by NVRTC for the specialised pass kernels, where no standard header
// exists: the host-only part is skipped there.
#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef signed char int8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#else
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tqs.h"
#endif

namespace tqs {

constexpr int kThreads = 256;      // threads per CTA of every state kernel
constexpr int kMaxTile = 13;       // largest shared-memory tile (2^13 amplitudes)
constexpr int kMaxGamma = 8;       // sampler group = up to 2^8 consecutive outcomes
constexpr int kProgChunkBytes = 6144;  // pass-program bytes staged in shared memory at a time
constexpr int kNoiseStage = 4096;      // noise bytes of a node staged in shared memory
constexpr uint32_t kDomNoise = 1, kDomMeas = 2, kDomRead = 3, kDomKraus = 4;

// ---------------------------------------------------------------------------
// Device-visible plan records
// ---------------------------------------------------------------------------
enum Op : uint8_t { OP_NOP = 0, OP_DENSE1 = 1, OP_DENSE2 = 2, OP_DIAG1 = 3, OP_DIAG2 = 4 };

// One gate (and the noise site that follows it) lowered for one pass.
struct Instr {
    uint8_t op;
    uint8_t j0, j1;      // tile positions of the gate qubits (dense ops)
    uint8_t p0, p1;      // physical bits of the gate qubits
    uint8_t np0, np1;    // physical bits of the noise site's qubits (a on np0, b on np1)
    uint8_t npaulis;     // 3 (one-qubit site) or 15 (two-qubit site)
    uint16_t site;       // site index relative to the level's first gate
    uint16_t pad;        // diagonal ops: bit k set iff factor k (G, a0, a1, c) != 1
    uint32_t gate;       // global gate index (row of the matrix tables)
};
static_assert(sizeof(Instr) == 16, "Instr layout");

// Pauli frame of a node at a pass boundary: logical psi(x) = i^phase * phi(x ^ mask)
// where phi is the stored vector (physical bit order).
struct NodeMeta {
    uint32_t mask;
    uint32_t phase;  // bits 0-1: i-power; bit 31 (entries 0..npass-1): the pass this entry opens
                     // holds a Pauli of this node
};
constexpr uint32_t kMetaNoisy = 0x80000000u;

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------------------
// Host-side circuit and plan
// ---------------------------------------------------------------------------
struct Gate {
    uint32_t kind, q0, q1;
    double theta;
    double m[32];  // interleaved complex matrix (2x2 or 4x4) in the local basis
};

struct Circuit {
    uint32_t n;
    std::vector<Gate> gates;
};

struct Noise {
    double p1, p2, pm;
    // non-unitary channels per qubit of a gate, in the order applied: thermal
    // relaxation's damping and dephasing (by the gate's arity), amplitude
    // damping, phase damping (rates; 0 = none)
    double ad = 0.0, pd = 0.0;
    double tr_g1 = 0.0, tr_l1 = 0.0, tr_g2 = 0.0, tr_l2 = 0.0;
    bool kraus() const { return ad > 0.0 || pd > 0.0 || tr_g1 > 0.0 || tr_l1 > 0.0 || tr_g2 > 0.0 || tr_l2 > 0.0; }
};

#endif  // __CUDACC_RTC__

// Compiled pass program: 16-byte aligned records walked in order by every
// thread of a CTA (uniform).  Record header, then a payload of complex values
// in the state's precision (R = float or double, C = complex of R):
//   REC_DENSE1  a=j b=p                 payload U[2x2]             noise site `site`
//   REC_DENSE2  a=j0 b=j1 c=p0 d=p1     payload U[4x4]             noise site `site`
//   REC_RUN     a..e = factor counts    payload G, then factors    sites [ibeg, iend) of the
//               of kinds A_FIXED, A_SLOT, C_FIXED, C_MIXED, C_SLOTS (in that order) for the
//               run of consecutive diagonal gates (and lazy SWAPs) it aggregates, then one
//               GateEnt (+ 4 factors) per gate of the run
// DENSE1 sets c = 1 when the matrix is real.  A factor record is an 8-byte FacHdr
// followed by its value at the next multiple of 8 (FP64: 32 bytes in all) or right
// after it (FP32: 16 bytes).  Diagonal values (G, the factors, the gate entries'
// four factors) are complex doubles in FP64 programs and phases in FP32 programs:
// one uint32 per value, the angle in units of 2^-32 turns (every diagonal gate
// kind has unit-modulus factors).
// A run's factors: the product over its gates of D = G * prod a_q^{x_q} *
// prod c_qr^{x_q x_r}, merged per qubit and per pair and classified by where
// the bits live (thread bit, register slot bit, outside the tile).
//   REC_FUSED   a=k (fused qubits)      no payload; ibeg/iend = the fused gates; `site` =
//               their first site; the 16 bytes after the header hold the k tile positions
//               (bytes 0..7), the k physical bits (bytes 8..15); the following 16 bytes hold
//               the float offset of the operand in PlanHost::fused (u32) and three zero words.
//               The kernels apply it as one 2^k x 2^k complex product on the tensor cores
//               (FP32 states only, k = t - 7 so that a tile has 128 columns).
//   REC_END     no payload: the end of the pass's program (every pass has one)
//   REC_KRAUS   a=j0 b=j1 c=p0 d=p1 e=qubits (1 or 2), no payload: the damping operators
//               chosen for this node after the previous gate, read per node from the
//               plan's operator buffer (2x2 on p0, then 2x2 on p1)
enum RecType : uint8_t { REC_DENSE1 = 1, REC_DENSE2 = 2, REC_RUN = 3, REC_FUSED = 4, REC_END = 5, REC_KRAUS = 6 };
enum FacKind : uint8_t {
    FAC_A_FIXED = 1,   // a^{x_p}, p a thread bit or outside the tile
    FAC_A_SLOT = 2,    // a^{x}, on slot bit s = j0 - 8
    FAC_C_FIXED = 4,   // c^{x_p0 x_p1}, neither on a slot bit
    FAC_C_MIXED = 5,   // c^{x_p0 x_s1}, p0 fixed, s1 = j1 - 8 a slot bit
    FAC_C_SLOTS = 7    // c^{x_s0 x_s1}, both slot bits
};
// FP32 programs: a REC_RUN record is RecHdr, then RunHdr32, then the factor
// entries {mask, phase} (8 bytes each): nbase entries for the thread's base
// phase, then ne[0] entries for slot 0's linear phase, ne[1] for slot 1, ...
// An entry applies to a thread iff its logical bits (physical bits XOR the
// frame mask) are 1 at every bit of `mask` (thread or outside-tile bits).
// Factors on slot bits alone are the same for every thread and are summed on
// the host into econst (linear, per slot) and gp (pairs, index hi(hi-1)/2+lo).
// Then padding to 16 bytes and the GateEnt list (phases) as for FP64.
constexpr uint32_t kMaxSlots = 5;
struct RunHdr32 {
    uint8_t nbase;
    uint8_t ne[kMaxSlots];
    uint16_t gused;            // pairs with a nonzero phase
    uint8_t eused;             // slots with a nonzero econst
    uint8_t pad[7];            // pad[0] = 1: only base entries (no slot term at all);
                               // pad[1] = all entries (nbase + sum of ne)
    uint32_t g0;               // global phase of the run
    uint32_t econst[kMaxSlots];
    uint32_t gp[kMaxSlots * (kMaxSlots - 1) / 2];
};
static_assert(sizeof(RunHdr32) == 80, "RunHdr32 layout");
struct RecHdr {
    uint8_t type, a, b, c;
    uint8_t d, e;
    uint16_t site;        // noise site (dense) / first site (run), level-relative
    uint32_t ibeg, iend;  // instruction range (the run's gates, for the per-gate fallback)
};
static_assert(sizeof(RecHdr) == 16, "RecHdr layout");
// A REC_RUN record ends with one GateEnt per gate of the run, each followed by
// the gate's four diagonal factors (G, a0, a1, c) in the state's precision: the
// path for nodes that hold a Pauli inside the run (the frame may change mid-run).
struct GateEnt {
    uint8_t op, fl, j0, p0;   // fl: bit k set iff factor k != 1 (as Instr::pad)
    uint8_t j1, p1, np0, np1;
    uint8_t npaulis, pad0, pad1, pad2;
    uint32_t site;
};
static_assert(sizeof(GateEnt) == 16, "GateEnt layout");
struct FacHdr {
    uint8_t kind, j0, p0, j1, p1, pad0, pad1, pad2;
};
static_assert(sizeof(FacHdr) == 8, "FacHdr layout");

#ifndef __CUDACC_RTC__
struct Pass {
    uint32_t level;
    uint32_t ibeg, iend;          // instruction range (global instruction list)
    uint32_t chunk_begin, chunk_end;  // program chunks (offsets in PlanHost::chunk_off)
    uint32_t fused_blocks;        // REC_FUSED records in the program
    uint32_t site_begin;          // first (lowest) site of the pass, relative to the level
    uint32_t t, L;                // tile width and number of contiguous low bits
    uint8_t tbits[kMaxTile];      // physical bit of each tile position (ascending)
    uint8_t hbits[32];            // remaining physical bits (ascending), n - t of them
    // Damping channels (a plan with Noise::kraus(): one gate per pass).  The
    // pass's epilogue writes the sums the choice after gate kout_gate needs
    // (kout_gate < 0: none); the REC_KRAUS record that opens the next pass
    // applies the chosen operators on kin_p0 (and kin_p1).
    int32_t kout_gate = -1;
    uint8_t kout_nq = 0, kout_p0 = 0, kout_p1 = 0;
    uint8_t kin_nq = 0, kin_p0 = 0, kin_p1 = 0;
};

struct Level {
    uint32_t g0, g1;              // gate range
    uint64_t arity;               // A_i
    uint64_t active;              // nodes simulated at this level
    uint64_t below;               // prod_{j>i} A_j
    uint32_t pass_begin, pass_end;
    std::vector<uint8_t> perm;    // logical qubit -> physical bit after this level
};

#endif  // __CUDACC_RTC__

// Measurement layout of the final pass: outcome y (logical) is grouped in blocks
// of 2^gamma consecutive values whose low gamma logical bits all lie in the tile.
struct SamplerLayout {
    uint32_t gamma;
    uint64_t groups;               // 2^(n - gamma) block sums per leaf
    uint8_t phys_of_logical[32];   // P[q]
    uint8_t rank_pos[kMaxTile];    // tile position of logical rank r (ascending logical bit)
    uint8_t rank_q[kMaxTile];      // logical bit of rank r
    uint8_t logical_of_hbit[32];   // logical bit of each non-tile physical bit
    int8_t rank_of_logical[32];    // rank within the tile, or -1 if the bit is not in the tile
};

#ifndef __CUDACC_RTC__
struct PlanHost {
    uint32_t n;
    tqs_precision prec;
    tqs_mode mode;
    uint64_t shots;
    std::vector<Level> levels;
    std::vector<Pass> passes;
    std::vector<Instr> instrs;       // per pass in site order (the noise kernel's table)
    std::vector<Instr> prog_instrs;  // per pass in program order (diagonal gates sunk)
    std::vector<double> mats64;    // 32 doubles per gate
    std::vector<float> mats32;     // 32 floats per gate
    std::vector<uint8_t> prog;     // compiled pass programs (state precision), all passes
    std::vector<uint32_t> chunk_off; // chunk boundaries into prog (chunk c = [off[c], off[c+1]))
    std::vector<float> fused;        // fused-gate operands (TF32 hi/lo, tensor-core B layout)
    uint32_t fused_k = 0;            // qubits per fused gate in this plan (0: none)
    bool fuse = false;               // FP32: fuse dense gate blocks onto the tensor cores
    uint64_t thr1, thr2, thrm;     // floor(p * 2^32)
    SamplerLayout samp;
    uint32_t tile_max;
    // damping channels: rates after a one-qubit (krate[0]) and a two-qubit gate
    // (krate[1]), per qubit in the order applied: thermal damping, thermal
    // dephasing, amplitude damping, phase damping
    bool kraus = false;
    double krate[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
};

// Host planning (planner.cpp)
std::string validate_and_build_circuit(uint32_t n, const tqs_gate *gates, size_t ng, Circuit &out);
void gate_matrix(uint32_t kind, double theta, const double *mat, double *out);
bool is_two_qubit(uint32_t kind);
bool is_diagonal(uint32_t kind);
std::string partition(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o,
                      std::vector<uint64_t> &arity, std::vector<uint32_t> &split);
std::string build_plan(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o,
                       const std::vector<uint64_t> &arity, const std::vector<uint32_t> &split,
                       PlanHost &p);
uint64_t threshold32(double p);

// ---------------------------------------------------------------------------
// Kernel launchers (kernels.cu; the pass kernel itself is in pass_kernel.cuh).
// All return the cudaError_t of the launch as int.
// ---------------------------------------------------------------------------
struct DevTables {
    const Instr *instr;
    const void *mats;          // double[32*G] or float[32*G] by precision
    const uint32_t *pass_site_begin;  // per global pass: first site (level-relative)
};

struct NoiseLaunch {
    const Instr *instr;        // the level's instructions (one per site, in order)
    uint32_t sites;            // sites in the level
    const uint32_t *pass_start;// device: first table entry of each pass (the level's instruction
                               // table runs in pass order), npass+1 entries
    uint32_t npass;
    uint64_t node_lo, nnodes;  // global ids [node_lo, node_lo + nnodes)
    const NodeMeta *parent_meta;  // nullptr for level 0
    uint32_t parent_stride;    // NodeMeta entries per parent slot
    uint32_t parent_end;       // index of the parent's final meta
    uint64_t parent_lo, arity;
    uint8_t *noise_out;        // [slot][sites]
    NodeMeta *meta_out;        // [slot][npass + 1]
    const uint64_t *seed_dev;  // when non-null the seed is read here (graph replays)
    uint64_t seed, thr1, thr2;
};
int launch_noise(const NoiseLaunch &a, void *stream);

#endif  // __CUDACC_RTC__

enum PassMode { MODE_STORE = 0, MODE_SUMS = 1, MODE_SAMPLE = 2 };

#ifndef __CUDACC_RTC__

struct PassLaunch {
    int mode;
    int fp64;
    const void *in;            // nullptr = synthesize |0...0>
    int in_from_parent;        // 1: input slot = node / arity - parent_lo, 0: own slot
    void *out;                 // STORE output states
    uint64_t state_elems;      // 2^n
    uint64_t node_lo, parent_lo, arity;
    uint32_t nnodes;
    const Instr *instr;
    uint32_t ibeg, iend;
    const uint8_t *prog;
    const uint32_t *chunk_off;
    uint32_t chunk_begin, chunk_end;
    uint32_t n, t, L;
    uint8_t tbits[kMaxTile];
    uint8_t hbits[32];
    const void *mats;
    const uint8_t *noise;
    uint32_t sites;
    const NodeMeta *meta;
    uint32_t meta_stride, pass_local;
    double *S;                 // SUMS / SAMPLE block sums
    const SamplerLayout *samp; // copied by value into the kernel parameters
    unsigned long long *counts;
    const uint64_t *seed_dev;  // when non-null the seed is read here (graph replays)
    uint64_t seed, thrm;
    const float *fused;        // fused-gate operands (device), nullptr when the pass has none
    uint32_t fused_k;          // qubits per fused gate (0: none)
    unsigned int *err;         // device error words: [0] bits (1 = a bounded tensor-core wait gave up,
                               // 2 = a fused record reached a kernel without the tensor-core path,
                               // 4 = an index check failed), [1] check code, [2] offending value
    uint32_t dbg;              // kDbgBounds | kDbgFaultTimeout
    uint64_t in_slots, out_slots;  // state slots of the input and output buffers (index checks)
    // damping channels: the epilogue writes, per tile, the four sums of |a|^2 by
    // the logical values of bits kp0 (low) and kp1 to ksum[slot][tile][4] (FP64;
    // nullptr = no sums); REC_KRAUS records read the node's operators from kmat
    double *ksum;
    const void *kmat;          // [slot][8] complex in the state's precision (2x2 on p0, 2x2 on p1)
    uint32_t knq, kp0, kp1;
    void *spec_fn;             // a kernel specialised for this pass and mode (specialize.h), or nullptr
};
#endif  // __CUDACC_RTC__
constexpr uint32_t kDbgBounds = 1u, kDbgFaultTimeout = 2u;
#ifndef __CUDACC_RTC__
int launch_pass(const PassLaunch &a, void *stream);

// The damping choices after one gate for `nnodes` nodes: sums the per-tile
// |a|^2 sums in a fixed order, draws and decides each channel in turn (the
// trajectory step of Sec. 4.3) and writes each node's 2x2 operators.
struct KrausLaunch {
    const double *ksum;        // [slot][tiles][4]
    uint64_t tiles;
    void *kmat;                // [slot][8] complex (state precision)
    int fp64;
    uint64_t node_lo, nnodes;
    const uint64_t *seed_dev;  // when non-null the seed is read here (graph replays)
    uint64_t seed;
    uint32_t gate, nq;
    double rate[4];            // thermal damping, thermal dephasing, amplitude damping, phase damping
};
int launch_kraus(const KrausLaunch &a, void *stream);
// Sets the shared-memory limits of every kernel variant (call before a stream capture).
int prepare_kernels();

int launch_fill_u64(unsigned long long *p, uint64_t n, void *stream);

// Fidelity of a histogram against the ideal state (FP64 reductions on device).
// ideal: stored physical-order ideal state; perm: logical -> physical.
int launch_fidelity(const void *ideal, int fp64, const unsigned long long *counts, uint32_t n,
                    const uint8_t *perm_dev, uint64_t shots, double *out3, void *stream);
#endif  // __CUDACC_RTC__

}  // namespace tqs
