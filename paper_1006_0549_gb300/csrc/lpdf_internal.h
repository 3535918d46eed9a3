// Internal structures of liblpdf (shared by the host API and the kernels of this library only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <mutex>
#include <vector>

#include "lpdf.h"

namespace lpdf {

constexpr int kHopCap = 64;
constexpr int kReflCap = 8;    // wall mirrorings of one particle in one step (edge walls)
constexpr int kMaxNS = LPDF_MAX_SCALARS;
// Moment sums are accumulated as 64-bit fixed point with 32 fractional bits: integer addition
// is associative, so the sums do not depend on the order in which CTAs and warps add them.
constexpr double kFixScale = 4294967296.0;      // 2^32
constexpr float kFixLimit = 1.0e9f;             // |partial| above this sets the overflow bit

inline int nfields(int ns) { return 22 + ns; }
inline int nfields_padded(int ns) { return (22 + ns + 3) / 4 * 4; }
inline int nquant(int ns) { return 11 + 2 * ns; }

// Device mesh. Per element: corner coordinates, centroid x, 1/(2 area), neighbours, node ids.
struct DevMesh {
    int n_nodes = 0, n_tri = 0;
    float x0 = 0, x1 = 0, y0 = 0, y1 = 0, period = 0;
    int periodic = 0;
    float4* ex = nullptr;     // (x0, x1, x2, centroid x)
    float4* ey = nullptr;     // (y0, y1, y2, 1 / (2 area))
    int4* en = nullptr;       // (nbr0, nbr1, nbr2, 0): neighbour across edge k, -1 = wall
    int4* ev = nullptr;       // (node0, node1, node2, 0): geometric node ids (node-field rows)
    int4* em = nullptr;       // (master0, master1, master2, 0): statistics node ids
    int* master = nullptr;    // n_nodes
    // affine barycentrics relative to vertex 0: lambda_1 = b1 dx + g1 dy, lambda_2 = b2 dx + g2 dy,
    // lambda_0 = 1 - lambda_1 - lambda_2, (dx, dy) = p - vertex 0
    float4* ea = nullptr;     // (x_v0, y_v0, b1, g1)
    float4* eb = nullptr;     // (b2, g2, centroid x, 0)
    double4* ec = nullptr;    // (b1, g1, b2, g2) in FP64: the barycentric combination of the moment sums
    // the walk's fast test reads one 64-byte record per element: ea, eb and en side by side
    // (one cache line instead of three), the fourth float4 unused
    float4* ew = nullptr;
    // several independent meshes in one (lpdf_mesh_load_multi): the component of every element
    // and each component's half-open frame [x0, x1) x [y0, y1); n_comp = 1 leaves both NULL
    int n_comp = 1;
    int* ecomp = nullptr;
    float4* cframe = nullptr;
    // 0: every wall edge lies on the frame's sides (walls are handled by mirroring at the frame);
    // 1: walls of any shape, mirrored across the wall edge through which the walk leaves
    int edge_walls = 0;
};

// per-component Philox key and scalar sources of a multi-component ensemble
// src_box: x0, x1, y0, y1 bounding every source disc, rounded outward to FP32 (empty without
// sources); a position outside it is outside every disc in the FP32 test as well
struct CompParams {
    uint32_t key0, key1;
    int n_src, pad;
    float src_box[4];
    float src_x[LPDF_MAX_SOURCES], src_y[LPDF_MAX_SOURCES], src_r[LPDF_MAX_SOURCES];
    int src_alpha[LPDF_MAX_SOURCES];
};

struct StepParams {
    float dt, sdt, s2nu, nu2, C3, C4, half_cphi, lid_u;
    uint32_t key0, key1;
    uint32_t step_lo, step_hi;
    int n_src;
    float src_box[4];
    float src_x[LPDF_MAX_SOURCES], src_y[LPDF_MAX_SOURCES], src_r[LPDF_MAX_SOURCES];
    int src_alpha[LPDF_MAX_SOURCES];
    const CompParams* comp;   // per component (multi-component meshes), else NULL
    const unsigned long long* step_dev;   // if set, the step number is *step_dev + step_add
    unsigned step_add;
    const float* beta;        // IECM: n_nodes x 3 ns conditional-mean slopes, else NULL (IEM)
    float react_k;            // reactive source psi_a + psi_b -> psi_p (none when <= 0)
    int react_a, react_b, react_p;
    int moment_sums;          // 0: FP32 partial sums; 1: compensated (lpdf_params.moment_sums)
};

struct DevState {
    float *x, *y, *u, *v, *w, *om, *psi;   // psi: ns rows of `cap` floats
    int* elem;
    uint32_t* pid;
    int64_t n, cap;
};

// Status words (device): [0] error bits, [1] lost count, [2] one lost pid, [3] total hops
enum : unsigned { kErrLost = 1u, kErrNonFinite = 2u, kErrOverflow = 4u, kErrTimeout = 8u, kErrCheck = 16u };

// Launchers (lpdf_kernels.cu)
cudaError_t launch_pdf_step(const DevMesh& m, const DevState& s, int ns, const float* fields,
                            const StepParams& p, unsigned long long* node_acc, unsigned long long* status,
                            cudaStream_t st);
// particle layout of an initialisation: component c holds particles [pbase[c], pbase[c + 1]),
// ppe[c] per element of its elements (from tri_off[c]); Philox key (key[2c], key[2c + 1])
struct InitLayout {
    const long long* pbase;
    const int* ppe;
    const int* tri_off;
    const uint32_t* key;
    int n_comp;
};
cudaError_t launch_particles_init(const DevMesh& m, const DevState& s, int ns, const InitLayout& L, int64_t P,
                                  const float* node_init, int m_erlang, unsigned long long* status, cudaStream_t st);
cudaError_t launch_grid_statistics(const DevMesh& m, int ns, const unsigned long long* node_acc, double* out,
                                   int raw, cudaStream_t st);

// scratch of the element re-bucketing: counts, cursors, bucket starts (E+1 buckets), permutation
struct SortScratch {
    int* cnt = nullptr;
    int* cursor = nullptr;
    int* start = nullptr;
    int* perm = nullptr;
};
cudaError_t launch_sort(const DevMesh& m, const DevState& s, int ns, const DevState& dst, SortScratch& w,
                        unsigned long long* status, cudaStream_t st);

// scratch of the step pipeline (lpdf_pipeline.cu)
struct PipeScratch {
    int* perm = nullptr;         // the current buffer in element order (the next step's gather order)
    int* perm_new = nullptr;     // written by the step: the next buffer in element order
    uint16_t* rrank = nullptr;   // per particle: (record slot << 8) | rank within its block's record
    int* rec_key = nullptr;      // per block record (block * 256 + slot): element, count, offset
    int* rec_cnt = nullptr;
    int* rec_off = nullptr;
    int* nrec = nullptr;         // records per block
    int* kwork = nullptr;        // 3 (E + 1) + 1: particles, records and cursors per element; K1's chunk counter
    int* kstart = nullptr;       // E + 1: bucket starts
    int* krstart = nullptr;      // E + 1: record-list starts
    int* klist = nullptr;        // records grouped by element, then in block order
    int* klist2 = nullptr;
    int* scan_part = nullptr;    // 2 x 4096 scan tile totals
    float* efields = nullptr;    // n_tri x 3 x nfp: node fields in element form
};
// ev (may be NULL): 4 events recorded before the advance kernel, after it, after the re-bucketing
// kernels and after the moments kernel
// launch configuration of the step's kernels (lpdf_ctx_autotune); every choice gives
// bit-identical results. adv: advance kernel 0 = 256 threads, >= 4 CTAs/SM; 1 = 128, >= 10,
// persistent grid; 2 = 128, >= 8; 3 = 256, >= 4, persistent; 4 = 64, >= 18, persistent; 5 = 128,
// >= 10, persistent, warps taking 64-particle chunks from a counter. mom: moments kernel
// 0 = 256 threads, >= 2 CTAs/SM; 1 = 128, >= 4; 2 = 512, >= 1; 3 = 256, >= 3.
struct StepTune {
    int adv = 0, mom = 0;
};
constexpr int kAdvVariants = 6, kMomVariants = 4;
cudaError_t launch_pdf_step_pipeline(const DevMesh& m, const DevState& cur, const DevState& nxt, int ns,
                                     const float* fields, const StepParams& p, PipeScratch& w,
                                     unsigned long long* node_acc, unsigned long long* status, cudaStream_t st,
                                     const cudaEvent_t* ev, const StepTune& tune,
                                     unsigned long long* flux_acc = nullptr);
cudaError_t launch_iota(int* p, int64_t n, cudaStream_t st);
// scalar fluxes per node (raw sums or covariances; n_nodes x 3 ns FP64) from the fixed-point sums
cudaError_t launch_flux_statistics(const int* master, int n_nodes, int ns, const unsigned long long* node_acc,
                                   const unsigned long long* flux_acc, double* out, int raw, cudaStream_t st);
// beta_a = R^-1 c_a per node (n_nodes x 3 ns FP32)
cudaError_t launch_iecm_coefficients(int n_nodes, int ns, const double* stats, const double* flux, float* beta,
                                     cudaStream_t st);
// SMs of the current device (queried once; call it before a stream capture)
int sm_count();
// *c = set (add = 0) or *c += add, one thread
cudaError_t launch_step_counter(unsigned long long* c, unsigned long long set, unsigned long long add, cudaStream_t st);

// tensor-core GEMM tile (lpdf_mlp.cu): D = A B^T, BF16 operands, FP32 result
cudaError_t launch_tc_gemm(const void* A, const void* B, float* D, int M, int N, int K, unsigned* error,
                           cudaStream_t st);

// P1 finite-element tables of the gridpoint solve (lpdf_solve.cu), built once per mesh.
// DOFs are the geometric nodes with periodic partners merged (numbered in node order).
struct Fem {
    static constexpr int kWorkPerDof = 65;     // FP64 scratch per DOF
    static constexpr int kDotBlocks = 1024;    // partial sums of one dot product
    int ndof = 0, nnz = 0, E = 0, N = 0;
    int* dof = nullptr;          // geometric node -> DOF
    int* dof_node = nullptr;     // DOF -> its master node (statistics row)
    int* edof = nullptr;         // 3 DOFs per element
    double* area = nullptr;      // per element
    double* grad = nullptr;      // 6 per element: grad of the 3 shape functions
    int* de_ptr = nullptr;       // DOF -> incident (element, corner) pairs e*3 + a (CSR)
    int* de_el = nullptr;
    double* darea = nullptr;     // sum of the areas of the incident pairs
    int* row = nullptr;          // DOF x DOF matrix pattern (CSR)
    int* col = nullptr;
    int* cptr = nullptr;         // CSR entry -> element-matrix contributions e*9 + a*3 + b
    int* cel = nullptr;
    double* Mval = nullptr;      // consistent mass matrix
    double* Kval = nullptr;      // stiffness matrix (unit coefficient)
    double* Aval = nullptr;      // M + L^2 K of the current solve
    unsigned char* wall = nullptr;
    double* normal = nullptr;    // inward unit normal per wall DOF
    double* work = nullptr;      // kWorkPerDof * ndof + 16 * E doubles
    double* part = nullptr;      // 12 * kDotBlocks: partial sums of up to three 4-vector dot products
    double* scal = nullptr;      // CG scalars (device)
    double* scal_host = nullptr; // pinned copy
    bool has_wp = false;         // the scratch holds a previous relaxation / pressure solution
    bool has_p = false;
    // wall distance of every geometric node (inputs of the learned surrogate)
    double* xy = nullptr;        // 2 per geometric node
    double* seg = nullptr;       // 4 per wall edge: (xa, ya, xb, yb)
    int* segn = nullptr;         // 2 per wall edge: its geometric end nodes a, b (grouped by component)
    int* seg_off = nullptr;      // per component: its wall edges [seg_off[c], seg_off[c + 1])
    int* ncomp = nullptr;        // component of every geometric node
    int nseg = 0, n_comp = 1;
    double period = 0.0;         // x period (0: none)
    // CUDA graphs of kCheckEvery CG iterations, one per call site (its matrix, diagonal, solution
    // and scratch pointers, component count and wall mask)
    struct CgGraph {
        const void* key[4];
        int nv, mask;
        cudaGraphExec_t exec;
    };
    std::vector<CgGraph> cg_graphs;
    cudaStream_t capture_stream = nullptr;
    double* wdist = nullptr;     // per geometric node, filled on first use: distance to the wall,
    int* wseg = nullptr;         //   the wall edge of the nearest wall point
    double* wt = nullptr;        //   and its position on that edge (0 at a, 1 at b)
    bool has_wdist = false;
};
cudaError_t fem_build(const double* node_xy, int n_nodes, const int32_t* tri, int n_tri, const int32_t* tag,
                      const std::vector<int32_t>& master, const std::vector<int32_t>& node_comp, double period,
                      Fem** out);
void fem_free(Fem* F);
// statistics (n_nodes x (11 + 2 ns), lpdf_grid_statistics raw = 0) -> node fields; iters[2];
// cudaErrorNotReady when a CG did not converge within maxit. With surr != NULL (n_nodes x 16
// standardised surrogate outputs, standardisation block surr_norm) the relaxation solve is
// replaced by the surrogate's G_ij and C_0 epsilon.
cudaError_t node_fields_solve(Fem& F, const double* stats, const lpdf_params& P, float* out, double tol,
                              int maxit, int* iters, cudaStream_t st, const float* surr = nullptr,
                              const float* surr_norm = nullptr);
// per geometric node: the 8 surrogate inputs (feat, n_nodes x 8) and, when fields != NULL, the 7
// targets taken from those node fields (tgt, n_nodes x 7)
cudaError_t surrogate_features(Fem& F, const double* stats, int ns, const float* fields, double C0, float* feat,
                               float* tgt, cudaStream_t st);
// out2 = {sum (a - b)^2, sum b^2} over the G_ij and C_0 epsilon columns of two node-field tables
cudaError_t fields_compare(const float* a, const float* b, int n_nodes, int nfp, double* out2, cudaStream_t st);

// the learned surrogate network (8 -> 128 -> 128 -> 128 -> 7, tanh, BF16 operands)
namespace mlp {
constexpr int kIn = 8, kInP = 16, kH = 128, kOut = 7, kOutP = 16;
// FP32 master parameters, padded: W1[128][16] (inputs 8..15 zero), b1[128], W2[128][128], b2[128],
// W3[128][128], b3[128], W4[16][128] (rows 7..15 zero), b4[16]
constexpr int oW1 = 0, ob1 = oW1 + kH * kInP, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + kH * kH,
              oW4 = ob3 + kH, ob4 = oW4 + kOutP * kH, kParams = ob4 + kOutP;
// BF16 packs: row-major [out][in] for the forward, [in][out] for the backward
constexpr int pW1 = 0, pW2 = pW1 + kH * kInP, pW3 = pW2 + kH * kH, pW4 = pW3 + kH * kH, pT2 = pW4 + kOutP * kH,
              pT3 = pT2 + kH * kH, pT4 = pT3 + kH * kH, kPack = pT4 + kH * kOutP;
// per-CTA gradient partials: W^T layouts [in][out] and the biases
constexpr int gW1 = 0, gW2 = gW1 + kInP * kH, gW3 = gW2 + kH * kH, gW4 = gW3 + kH * kH, gb1 = gW4 + kH * kOutP,
              gb2 = gb1 + kH, gb3 = gb2 + kH, gb4 = gb3 + kH, kPart = gb4 + kOutP;
// standardisation block: feature means and deviations, loss weights, target means and deviations
constexpr int nFM = 0, nFS = nFM + kIn, nW = nFS + kIn, nTM = nW + kOut, nTS = nTM + kOut, kNorm = nTS + kOut;
}  // namespace mlp
cudaError_t mlp_configure();
cudaError_t launch_mlp_forward(const float* feat, int64_t B, const float* P, const void* pack, const float* norm,
                               float* out, float* out_user, void* act, unsigned* error, cudaStream_t st);
// per-CTA partials into part ((B + 127) / 128 x kPart), then their sum in CTA order into grad
cudaError_t launch_mlp_backward(const float* feat, const float* tgt, int64_t B, const void* pack, const float* norm,
                                const float* out, const void* act, float* part, float* grad, unsigned* error,
                                cudaStream_t st);
cudaError_t launch_mlp_adam(float* P, const float* grad, float* m, float* v, float lr, int step, void* pack,
                            cudaStream_t st);
cudaError_t launch_mlp_loss(const float* out, const float* tgt, int64_t B, const float* norm, double* loss,
                            cudaStream_t st);
// feature and target means and deviations of a data set into norm (weights untouched)
cudaError_t launch_mlp_fit_norm(const float* feat, const float* tgt, int64_t B, float* norm, cudaStream_t st);

// the gridpoint tables of a mesh, built on first use (LPDF_OK or an error code with the message set)
int mesh_fem(const struct ::lpdf_mesh* mesh, Fem** out);

StepParams make_step_params(const lpdf_params& p, const struct ::lpdf_mesh* m, uint64_t step);
// records the calling thread's error message (lpdf_last_error) and returns `code`
int lpdf_set_error(int code, const char* fmt, ...);

}  // namespace lpdf

// Opaque handles of the C ABI (defined here so that every translation unit of the library
// can reach the device tables).
struct lpdf_mesh {
    lpdf::DevMesh d;
    std::vector<int32_t> nbr;      // host copy, 3 per element
    std::vector<int32_t> master;   // host copy
    std::vector<double> node_xy;   // host copies of the input (for the gridpoint solve)
    std::vector<int32_t> tri, tag;
    std::vector<int32_t> node_comp;  // component of every node
    std::vector<int32_t> elem_comp;  // component of every element
    double period = 0.0;             // x period (0: walls)
    double box[4];
    int device;
    mutable std::mutex fem_mutex;
    mutable lpdf::Fem* fem = nullptr;   // built by the first lpdf_elliptic_relax_solve call
};

struct lpdf_ctx {
    const lpdf_mesh* mesh;
    lpdf_params params;
    lpdf::DevState s;                         // current particle state
    lpdf::DevState s2;                        // second buffer (written by the step and the re-bucketing)
    lpdf::SortScratch sort;
    lpdf::PipeScratch pipe;
    unsigned long long* node_acc = nullptr;   // n_nodes x nq fixed-point sums
    unsigned long long* flux_acc = nullptr;   // n_nodes x 3 ns fixed-point scalar-flux sums (IECM)
    const float* iecm_beta = nullptr;         // lpdf_ctx_set_iecm
    unsigned long long* status = nullptr;     // 4 words
    int ns;
    int64_t nsteps = 0;                       // pdf_step calls so far
    // per-kernel timing (lpdf_ctx_set_timing): event quadruples of the recorded steps
    lpdf::StepTune tune;                      // lpdf_ctx_autotune's choice
    lpdf::CompParams* comp = nullptr;         // per component (multi-component meshes), device
    std::vector<lpdf::CompParams> comp_host;
    bool comp_set = false;                    // lpdf_ctx_set_components was called
    // the last initialisation layout (device): pbase, ppe, tri_off, keys
    long long* init_pbase = nullptr;
    int* init_ppe = nullptr;
    int* init_toff = nullptr;
    uint32_t* init_key = nullptr;
    const float* graph_state[2] = {nullptr, nullptr};   // the buffer and order each graph was captured on
    const int* graph_perm[2] = {nullptr, nullptr};
    int graph_next = 0;                       // the slot the next capture replaces
    cudaStream_t graph_stream = nullptr;
    // CUDA graphs of two consecutive steps (lpdf_pdf_steps), for the fields pointer they captured
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    const float* graph_fields[2] = {nullptr, nullptr};
    unsigned long long* step_dev = nullptr;   // the step number the graph's kernels read
    bool timing = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::array<cudaEvent_t, 4>> ev_pending;
};
