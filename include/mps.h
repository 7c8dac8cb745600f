/*
 * mps.h - C ABI of the GB300 (sm_103a) engine for the time-dependent
 * matrix-product-state (MPS) simulation of quantum circuits.
 *
 * Method: A. SaiToh, "A Multiprecision Matrix Calculation Library and Its
 * Extension Library for a Matrix-Product-State Simulation of Quantum
 * Computing" (2011), Sec. 3. The state is held in the Vidal form of Eq. (1):
 * site tensors Gamma_s (the paper's Q_s, 2 x m_{s-1} x m_s complex numbers)
 * and bond vectors Lambda_s (the paper's V_s, the Schmidt coefficients of the
 * cut (0..s)|(s+1..n-1), Eq. (2)). A gate on consecutive qubits rewrites only
 * the tensors it touches (Sec. 3.1); small Schmidt coefficients are truncated.
 *
 * Conventions shared by every call:
 *  - Complex numbers are complex128: two doubles (real, imaginary), interleaved.
 *  - A k-qubit gate or operator is a 2^k x 2^k row-major complex128 matrix.
 *    Its row/column index is sum_j b_{site+j} 2^{k-1-j}: the FIRST acted-on
 *    qubit is the MOST significant bit. (The Sec. 3.2 example, CNOT on qubits
 *    0 and 2 with 0 as control, fixes this order.)
 *  - Bond b (0 <= b <= n-2) sits between qubits b and b+1.
 *  - Host pointers passed in are read before the call returns; the library
 *    never keeps or frees caller memory. Output buffers are caller-allocated.
 *  - Every entry point returns an mps_status. Argument errors are reported
 *    synchronously and leave the state untouched. Errors found on the device
 *    (for instance a Jacobi SVD that did not converge) are recorded in a
 *    device status word and reported by the next call that synchronises
 *    (mps_sync, readouts, exports); the gate that failed leaves its tensors
 *    unchanged. mps_last_error() returns a message for the calling thread.
 *  - Calls on one handle are issued on that handle's CUDA stream in order;
 *    a handle must not be used from two threads at once.
 */
#ifndef PAPER_1111_3124_GB300_MPS_H
#define PAPER_1111_3124_GB300_MPS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mps_state* mps_handle;

typedef enum {
  MPS_OK = 0,
  MPS_ERR_ARG = -1,          /* bad argument (null pointer, range, shape)    */
  MPS_ERR_NOMEM = -2,        /* device or pinned-host allocation failed      */
  MPS_ERR_CUDA = -3,         /* a CUDA runtime call failed                   */
  MPS_ERR_NOCONVERGE = -4,   /* Jacobi SVD hit its sweep limit               */
  MPS_ERR_TIMEOUT = -5,      /* a bounded device wait ran out                */
  MPS_ERR_NOT_UNITARY = -6,  /* ||U^H U - I||_max > 1e-10                    */
  MPS_ERR_TOO_LARGE = -7     /* request exceeds a stated size limit          */
} mps_status;

/* Arithmetic used for the dense contractions of the gate update. */
typedef enum {
  MPS_PREC_FP64 = 0,   /* native binary64 on the CUDA cores                   */
  MPS_PREC_SPLIT = 1   /* binary64-accurate products from sliced bf16 tensor-
                          core products (Ozaki scheme); the SVD runs fp32
                          Jacobi sweeps, then binary64 Gram-polish steps on
                          split-precision Gram matrices (binary64 angles and
                          orthogonality test), the blocked binary64 sweeps
                          as the fallback                                    */
} mps_prec;

/* SVD of the gate update (mps_set_mode's svd_mode). */
typedef enum {
  MPS_SVD_JACOBI = 0,     /* full blocked one-sided Jacobi SVD                 */
  MPS_SVD_SKETCH_MLP = 1  /* rank predicted by an MLP (mps_set_predictor) sizes
                             a randomized range-finder sketch; the full Jacobi
                             SVD is the fallback when the sketch's residual
                             exceeds max(cutoff/100, Mw eps) ||theta||_F, and
                             is used directly when the sketch width would not
                             be well below full rank or would reach chi_max  */
} mps_svd_mode;

/* The rank predictor: a 16-64-1 tanh MLP in fp32 (no paper counterpart: the
 * learned part of this engine). Parameters (1153 floats): W1[64][16],
 * b1[64], w2[64], b2; y = b2 + sum_h w2[h] tanh(b1[h] + sum_i W1[h][i] x_i).
 * The target is log2(r) / 10 with r the rank a sketch must capture
 * (mps_diag's k_sketch). */
typedef struct mps_mlp* mps_mlp_handle;

/* Creates an MLP on the current device with Glorot-uniform weights drawn from
 * a generator seeded by `seed` and zero biases. */
int mps_mlp_create(unsigned long long seed, mps_mlp_handle* out);
int mps_mlp_destroy(mps_mlp_handle m);
/* Copies the 1153 parameters out (get, may be NULL) and/or in (set, may be
 * NULL; resets the optimizer state). Host pointers. */
int mps_mlp_params(mps_mlp_handle m, float* get, const float* set);
/* Y[b] = MLP(X[b]) for B samples; X is B x 16, host pointers. */
int mps_mlp_forward(mps_mlp_handle m, int B, const float* X, float* Y);
/* Mean squared error over the B samples and its gradient (1153 floats; NULL
 * to skip), by the hand-written backward kernel. Host pointers. */
int mps_mlp_loss_grad(mps_mlp_handle m, int B, const float* X, const float* T, float* loss, float* grad);
/* Trains with Adam (beta 0.9/0.999) on N samples (host X: N x 16, T: N) for
 * `epochs` shuffled passes of mini-batches of size `batch`; *loss receives the
 * mean batch loss of the last epoch. */
int mps_mlp_train(mps_mlp_handle m, int N, const float* X, const float* T, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss);

/* mps_create - Sec. 3.2 ("mps M(n)"): an n-qubit state |0...0>, i.e.
 * Gamma_s[0] = [[1]], Gamma_s[1] = [[0]], Lambda_b = [1].
 *   n        number of qubits, 1 <= n <= 4096
 *   chi_max  largest bond dimension kept after a gate, 1 <= chi_max <= 1024
 *            (device memory for the tensors is reserved at this capacity:
 *            n * 2 * chi_max^2 * 16 bytes)
 *   cutoff   truncation threshold (Sec. 3.1, "very small coefficients ... are
 *            truncated out"): after each split, the Schmidt values sigma_j
 *            with sigma_j <= cutoff * ||sigma||_2 are dropped, at most chi_max
 *            values are kept (ties broken by column index), at least one, and
 *            the kept values are renormalised to unit 2-norm. cutoff >= 0.
 *   out      receives the handle (set to NULL on error).
 * Errors: MPS_ERR_ARG, MPS_ERR_NOMEM, MPS_ERR_CUDA. */
int mps_create(int n, int chi_max, double cutoff, mps_handle* out);

/* Releases the handle and all device memory it owns. NULL is accepted. */
int mps_destroy(mps_handle h);

/* Makes every later call of this handle run on `cuda_stream` (a cudaStream_t
 * owned by the caller, e.g. a PyTorch stream). NULL restores the handle's own
 * stream. The caller keeps the stream alive while the handle uses it. */
int mps_set_stream(mps_handle h, void* cuda_stream);

/* Selects the arithmetic of later gate updates (prec = mps_prec). `slices` is
 * the number of bf16 slices per operand for MPS_PREC_SPLIT (0 = default 8,
 * range 3..8); it is ignored for MPS_PREC_FP64. `svd_mode` is an
 * mps_svd_mode; MPS_SVD_SKETCH_MLP needs a predictor (mps_set_predictor). */
int mps_set_mode(mps_handle h, int prec, int slices, int svd_mode);

/* mps_set_limits - the sweep limit of the binary64 blocked Jacobi SVD of
 * later gate updates (1 <= max_sweeps <= 60, default 60; the paper gives no
 * limit, this engine's reading of Sec. 3.1's SVD). An update that reaches it
 * without converging is left unapplied and reported as MPS_ERR_NOCONVERGE by
 * the next synchronising call. Errors: MPS_ERR_ARG. */
int mps_set_limits(mps_handle h, int max_sweeps);

/* mps_set_tuning - the launch shape of the split mode's fp32 sweeps per
 * working-matrix width Nw (the smaller dimension of theta; no paper
 * counterpart: chosen by measurement, see the package's tuner). Entry i
 * applies to Nw <= nw_max[i] (increasing; the last entry also covers larger
 * widths): f32_block[i] = 8 or 16 columns per block; f32_mode[i] = 0 launches
 * one round of block pairs at a time with the rotation in the pair kernel,
 * 1 does the same with the block rotations on the tensor cores (block width
 * 16 only), 2 runs every sweep of every task of the pass in one scheduled
 * launch (pairs taken in order as their inputs become final) of 256-thread
 * CTAs, 3 the same with 384-thread CTAs (fewer, faster pairs at a time). All
 * four compute the same rotations; 0 and 2 give identical results (3 sums
 * each Gram over a different grouping of rows). n = 0 restores the default
 * (16, mode 2). Host arrays. Errors: MPS_ERR_ARG. */
int mps_set_tuning(mps_handle h, int n, const int* nw_max, const int* f32_block, const int* f32_mode);

/* mps_debug_fail_alloc - test hook for the allocation-failure path (no paper
 * counterpart): the next `after` device or pinned-host allocations made by
 * the library succeed, the one after that is refused as if the device were out
 * of memory (the call that needed it returns MPS_ERR_NOMEM and leaves the
 * state as it was); after < 0 turns the hook off. Process-wide. */
int mps_debug_fail_alloc(long long after);

/* mps_debug_bounded_wait - test hook for the timeout path (no paper
 * counterpart): runs, on `stream`, the bounded mbarrier wait that the
 * tensor-core kernels use, on a barrier that nothing completes, with a limit
 * of limit_ms (0 < limit_ms <= 10000). The wait gives up, the kernel returns
 * with its error flag set and this call reports MPS_ERR_TIMEOUT. No copy or
 * product is in flight when it gives up, so the context stays usable.
 * Synchronises `stream`. Errors: MPS_ERR_ARG, MPS_ERR_NOMEM, MPS_ERR_CUDA,
 * MPS_ERR_TIMEOUT (the expected outcome). */
int mps_debug_bounded_wait(double limit_ms, void* stream);

/* mps_debug_mark_timed_out - test hook (no paper counterpart): marks the
 * handle as if a bounded wait of its split GEMM had run out. Every later
 * split-precision product of the handle is refused with MPS_ERR_TIMEOUT before
 * anything is launched, as after a real timeout (whose abandoned copies and
 * products leave the device state untrusted). */
int mps_debug_mark_timed_out(mps_handle h);

/* mps_reset - returns the state to |0...0> (same as a fresh mps_create). */
int mps_reset(mps_handle h);

/* mps_apply_gate - Sec. 3.1 / Sec. 3.2 ("applyU"): applies U in U(2^k),
 * k in {1,2,3}, to qubits site..site+k-1.
 *   k = 1: Gamma_site <- u Gamma_site on the physical index (no SVD). Single-
 *          qubit gates are held back and folded into the next multi-qubit
 *          gate touching the same qubit, or applied before any readout.
 *   k = 2: two-site update of Gamma_s, Lambda_s, Gamma_{s+1} (Sec. 3.1):
 *          theta = Lambda_{s-1} Gamma_s Lambda_s Gamma_{s+1} Lambda_{s+1}
 *          contracted with U, split by a one-sided Jacobi SVD, truncated
 *          (see mps_create), outer Lambdas divided back out.
 *   k = 3: three-site update (U(8) gates are elementary, Sec. 1, Sec. 3.1):
 *          one theta over three sites split by two successive SVDs.
 *   U      host pointer, 2^k x 2^k row-major complex128, copied before return.
 * Errors: MPS_ERR_ARG (k, site range, NULL), MPS_ERR_NOT_UNITARY. */
int mps_apply_gate(mps_handle h, int site, int k, const double* U);

/* mps_apply_gate_on - Sec. 3.2 ("applyU(U, q0, q1)", e.g. CNOT on qubits 0
 * and 2): a one- or two-qubit gate on any listed qubits. The first listed
 * qubit is the most significant bit of U's index, whatever the qubits' order.
 * Neighbours are one two-site update. At distance 2, route 0 embeds U as a
 * U(8) on (q, q+1, q+2) with the identity on the middle qubit (one three-site
 * update); otherwise SWAP updates carry the higher qubit next to the lower
 * one, U acts there, and SWAP updates carry it back (2 (d - 1) + 1 two-site
 * updates for distance d, each truncated as usual). route: 0 (embed at
 * distance 2, SWAPs beyond) or 1 (SWAPs always).
 * Errors: MPS_ERR_ARG, MPS_ERR_NOT_UNITARY. */
int mps_apply_gate_on(mps_handle h, int nq, const int* qubits, const double* U, int route);

/* mps_apply_layer - n_gates gates of the same size k on pairwise disjoint
 * qubit ranges, updated together in one batched pass (the gates of one
 * circuit layer commute, so the result equals applying them in any order).
 *   sites  host array of n_gates first sites
 *   Us     host array of n_gates gates, each 2^k x 2^k complex128, row-major,
 *          stored one after another
 * Errors: MPS_ERR_ARG (overlap, range, NULL), MPS_ERR_NOT_UNITARY. */
int mps_apply_layer(mps_handle h, int k, int n_gates, const int* sites, const double* Us);

/* mps_apply_layer_device - as mps_apply_layer, but the n_gates gates are read
 * from DEVICE memory (d_Us: n_gates x 2^k x 2^k complex128, row-major, on the
 * handle's device), so a caller whose gates are already resident in HBM pays
 * no host-to-device copy. The buffer must stay valid until the handle's stream
 * has executed this call. No unitarity check is made. Held-back single-qubit
 * gates on the touched qubits are applied first; k = 1 gates are applied at
 * once (not held back).
 *   sites  host array of n_gates first sites (pairwise disjoint ranges)
 * Errors: MPS_ERR_ARG. */
int mps_apply_layer_device(mps_handle h, int k, int n_gates, const int* sites, const double* d_Us);

/* mps_apply_layer_multi - gates of MANY independent MPS updated together:
 * the gate tasks of all handles share batched passes (largest problems
 * first, in passes whose workspace fits a fixed memory budget), which keeps
 * the GPU busy when each circuit alone has few or small gates.
 *   count     number of handles (>= 1), pairwise distinct, same device
 *   handles   the MPS; the work runs on handles[0]'s stream with its
 *             workspace and arithmetic mode; the other handles' streams are
 *             synchronised before and made to wait for the work after
 *   k         2 or 3 (all gates of the call have the same size)
 *   n_gates   per handle, the number of its gates (disjoint within a handle)
 *   sites     concatenation over handles of their first sites
 *   Us        concatenation of the gates, 2^k x 2^k complex128 row-major each
 * Errors: MPS_ERR_ARG, MPS_ERR_NOT_UNITARY (nothing applied). */
int mps_apply_layer_multi(int count, const mps_handle* handles, int k, const int* n_gates, const int* sites,
                          const double* Us);

/* mps_layer_features - the 16 predictor features of each of n_gates two-site
 * gates as they would be applied to the current state (nothing is applied):
 *   log2 chi_{s-1}/10, log2 chi_{s+1}/10, log2 chi_s/10, 4.5 e_p(U) (the
 *   entangling power, Zanardi-Zalka-Faoro 2000), ln of the 6 largest
 *   Lambda_{s-1} and of the 6 largest Lambda_{s+1}, each / 25, missing values
 *   padded with ln(max(cutoff, 1e-13))/25.
 *   X  host buffer of n_gates x 16 floats. Synchronises the stream. */
int mps_layer_features(mps_handle h, int k, int n_gates, const int* sites, const double* Us, float* X);

/* Attaches the rank predictor used when svd_mode is MPS_SVD_SKETCH_MLP (the
 * MLP must outlive its use; NULL detaches). */
int mps_set_predictor(mps_handle h, mps_mlp_handle m);

/* Counters of the sketch path since the handle's creation: gates whose SVD
 * was attempted by the sketch, sketches accepted, gates routed directly to
 * the full Jacobi SVD by the predictor. Any pointer may be NULL. */
int mps_sketch_stats(mps_handle h, long long* sketched, long long* accepted, long long* routed_full);

/* mps_amplitude - <bits|psi> = Gamma_0[b_0] Lambda_0 Gamma_1[b_1] ... Gamma_{n-1}[b_{n-1}]
 * (Eq. 1 evaluated at one basis state).
 *   bits  host array of n bytes, bits[q] in {0,1} is the value of qubit q
 *   out   host double[2] (real, imaginary)
 * Synchronises the stream. */
int mps_amplitude(mps_handle h, const unsigned char* bits, double* out);

/* mps_amplitudes - `count` amplitudes in one launch; bits is count x n bytes,
 * out is count x 2 doubles. Synchronises the stream. */
int mps_amplitudes(mps_handle h, int count, const unsigned char* bits, double* out);

/* mps_expectation - <psi|O|psi> / <psi|psi> for a k-qubit operator O acting on
 * qubits site..site+k-1 (k in {1,2,3}, same index convention as gates), by a
 * full transfer-matrix contraction of Eq. (1), exact for the stored tensors.
 *   out   host double[2]. Synchronises the stream. */
int mps_expectation(mps_handle h, int site, int k, const double* O, double* out);

/* mps_reduced_density - Sec. 3.2 ("RDO", the tracing-out operation): the
 * reduced density operator of the listed qubits, normalised to unit trace,
 * by a transfer-matrix contraction of Eq. (1) run from whichever end of the
 * chain keeps the environments smaller.
 *   qubits  host array of nq distinct qubit indices in any order; the first
 *           listed qubit is the most significant bit of rho's index (as in
 *           the Sec. 3.2 output |00><11|)
 *   nq      1 <= nq <= 12
 *   rho     host buffer of 2^nq x 2^nq complex128, row-major
 * The contraction holds 4^t x chi^2 entries after t listed qubits (chi the
 * bond it has reached); a request that would hold more than 2^27 entries in
 * one buffer is refused with MPS_ERR_TOO_LARGE. The working buffers are the
 * handle's (grown on demand, released by mps_destroy).
 * Errors: MPS_ERR_ARG, MPS_ERR_TOO_LARGE (nq > 12 or the size above),
 * MPS_ERR_NOMEM. Synchronises the stream. */
int mps_reduced_density(mps_handle h, const int* qubits, int nq, double* rho);

/* mps_sample - `count` bit strings drawn from |<b|psi>|^2 / <psi|psi> (the
 * measurement of every qubit in the computational basis, Eq. 1's amplitudes)
 * by sequential conditional sampling: qubit s of sample m is 0 when
 * u[m n + s] < p(b_s = 0 | b_0 .. b_{s-1}), else 1. The conditional weights
 * contract the sample's chosen prefix with right environments of the stored
 * tensors, so they are exact for a truncated (non-canonical) state too.
 *   u     host array of count x n uniforms in [0, 1) (the caller's random
 *         numbers: the same u always gives the same strings)
 *   bits  host array of count x n bytes, bits[m n + q] in {0, 1} is qubit q
 * Errors: MPS_ERR_ARG (u outside [0, 1)), MPS_ERR_NOMEM. Synchronises the stream. */
int mps_sample(mps_handle h, int count, const double* u, unsigned char* bits);

/* mps_pauli_expectations - <psi|P|psi> / <psi|psi> for `count` Pauli strings
 * P = P_0 (x) ... (x) P_{n-1}, each P_q one of I, X, Y, Z, by full
 * transfer-matrix contractions of Eq. (1) (exact for the stored tensors).
 *   paulis  host array of count x n characters from "IXYZ" (no terminators)
 *   out     host array of count x 2 doubles (real, imaginary)
 * Errors: MPS_ERR_ARG, MPS_ERR_NOMEM. Synchronises the stream. */
int mps_pauli_expectations(mps_handle h, int count, const char* paulis, double* out);

/* mps_get_schmidt - copies Lambda_bond (the Schmidt coefficients of the cut
 * after qubit `bond`, Eq. 2) into lambda (capacity chi_max doubles) and its
 * length into *len. Synchronises the stream. */
int mps_get_schmidt(mps_handle h, int bond, double* lambda, int* len);

/* mps_bond_dims - chi[b] = current dimension of bond b, b = 0..n-2 (n-1 ints).
 * Synchronises the stream. */
int mps_bond_dims(mps_handle h, int* chi);

/* mps_export - copies the state to host arrays.
 *   chi      n+1 ints: chi[0] = chi[n] = 1, chi[b+1] = dim of bond b
 *   gammas   concatenation over s of Gamma_s as [2][chi[s]][chi[s+1]]
 *            complex128 (may be NULL to query chi only)
 *   lambdas  concatenation over b = 0..n-2 of Lambda_b (may be NULL)
 * Synchronises the stream. */
int mps_export(mps_handle h, int* chi, double* gammas, double* lambdas);

/* mps_import - replaces the state with host arrays laid out as in mps_export.
 * Every chi entry must lie in [1, chi_max] and chi[0] = chi[n] = 1. */
int mps_import(mps_handle h, const int* chi, const double* gammas, const double* lambdas);

/* mps_diag - diagnostics of the last gate or layer call, one entry per gate in
 * call order (at most `cap` entries; *count receives how many exist):
 *   k[i]          new bond dimension (for k = 3: of the second split)
 *   discarded[i]  discarded weight sum_{dropped} sigma^2 / sum sigma^2
 *                 (k = 3: sum over both splits)
 *   sweeps[i]     Jacobi sweeps used (k = 3: both splits)
 *   k_sketch[i]   singular values above max(cutoff / 100, Mw eps) ||sigma||
 *                 (before the chi_max cap): the rank a randomized sketch of
 *                 this update must capture to be accepted (MPS_SVD_SKETCH_MLP);
 *                 the rank predictor is trained on it
 * Any output pointer may be NULL. Synchronises the stream. */
int mps_diag(mps_handle h, int cap, int* count, int* k, double* discarded, int* sweeps, int* k_sketch);

/* Per-kernel-class timing of later calls (not part of the method; used to
 * measure each kernel against its roofline). enable = 1 brackets every launch
 * of the classes below with CUDA events on the handle's stream and counts the
 * executed flops; enable = 0 stops; each call clears the counters.
 * Kernel classes: 0 = binary64 Jacobi pair rotations, 1 = binary64 theta
 * contraction, 2 = truncation and tensor rewrite (norms, truncate, emit),
 * 3 = split-precision products (tensor-core flops), 4 = fp32 Jacobi pair
 * rotations (split mode), 5 = split-mode element-wise steps (gate mix,
 * conversions, Newton-Schulz update, Gram-polish test, rotation generator and
 * Givens rotations). */
int mps_profile(mps_handle h, int enable);

/* Reads the counters of class `kernel`: summed launch durations in ms, the
 * number of launches, and the executed flops (binary64 flops for classes 0-2,
 * tensor-core flops for class 3). `launches_all` (may be NULL) receives the
 * number of kernels of every class launched since the last mps_profile call.
 * Synchronises the stream. */
int mps_profile_read(mps_handle h, int kernel, double* ms, long long* launches, double* flops,
                     long long* launches_all);

/* A recorded circuit: passes of gate updates over one or more MPS, replayed
 * as one CUDA graph (no paper counterpart: the batched, graph-captured form
 * of the Sec. 3.1 update; many circuits at once is the batched workload).
 * A program holds copies of its gates, the task tables of every pass and its
 * own workspace; it must be destroyed before its handles. */
typedef struct mps_program* mps_program_handle;

/* mps_program_create - records n_passes passes. Pass p applies n_gates[p]
 * gates of k[p] qubits (1, 2 or 3); gate g of the concatenation over passes
 * acts on handle handles[owners[g]] (owners may be NULL when count = 1) at
 * qubits sites[g] .. sites[g] + k - 1, and the gates of one pass are disjoint
 * within each handle. d_Us: DEVICE memory holding every gate, 2^k x 2^k
 * complex128 row-major, pass after pass (copied at creation). The work runs on
 * handles[0]'s stream with its arithmetic mode; k = 1 gates are applied as
 * they come (not held back).
 * The recording needs no host synchronisation at replay: grids are sized for
 * the bond bounds min(chi_max, 2 chi_l, 2 chi_r) that follow from every
 * handle's bonds at creation, the Jacobi sweep loops are conditional (while)
 * nodes whose continuation the device sets after each sweep (bounded by the
 * sweep limits), and the task tables are built once. Recording applies
 * nothing; held-back single-qubit gates of the handles are applied first.
 * Errors: MPS_ERR_ARG, MPS_ERR_NOMEM, MPS_ERR_CUDA. */
int mps_program_create(int count, const mps_handle* handles, int n_passes, const int* k, const int* n_gates,
                       const int* sites, const int* owners, const double* d_Us, mps_program_handle* out);

/* mps_program_run - replays the program on handles[0]'s stream, from the
 * handles' current states (the other handles' streams are ordered before and
 * after it). Every bond must be within the bound it had when the program was
 * recorded (true after mps_reset for a program recorded from |0...0>), else
 * MPS_ERR_ARG. Asynchronous: a deferred device error (MPS_ERR_NOCONVERGE on
 * handles[0]) surfaces at the next synchronising call. */
int mps_program_run(mps_program_handle p);

/* Two- and three-site updates a run of the program performs. */
int mps_program_updates(mps_program_handle p, long long* updates);

/* Releases the program after waiting for the device to finish its work. The
 * program's handles may be destroyed before or after it (a run needs them
 * alive). NULL is accepted. */
int mps_program_destroy(mps_program_handle p);

/* mps_sync - waits for the handle's stream and reports a deferred device
 * error (MPS_ERR_NOCONVERGE, MPS_ERR_TIMEOUT, MPS_ERR_CUDA), clearing it. */
int mps_sync(mps_handle h);

/* mps_gate2_update_noalloc - one two-site (U(4)) gate update, the same
 * computation as mps_apply_gate with k = 2, applied to tensors the caller
 * keeps in device memory, WITHOUT ALLOCATING ANYTHING. The paper has no
 * counterpart; it serves callers that cannot allocate device memory while
 * they run: programs whose allocator already holds the device's memory
 * budget, or loops that must not stall on cudaMalloc/cudaFree (both may
 * synchronise the whole device). Its working storage is a fixed file-scope
 * device array of about 520 KB, present on every device that loads this
 * library until the process exits; no cudaMalloc, cudaFree or allocating
 * library routine is called.
 *   d_gamma_l   Gamma_s,     [2][chi_max][chi_max] complex128, device, rewritten
 *   d_gamma_r   Gamma_{s+1}, same layout, device, rewritten
 *   d_lambda_l  Lambda_{s-1}, chi_max doubles, device ([1] at the left end)
 *   d_lambda_m  Lambda_s, chi_max doubles, device, rewritten
 *   d_lambda_r  Lambda_{s+1}, chi_max doubles, device ([1] at the right end)
 *   d_chi       3 ints on the device: chi_{s-1}, chi_s, chi_{s+1}, each in
 *               [1, chi_max]; chi_s is rewritten with the kept rank
 *   chi_max     capacity and truncation limit, 1 <= chi_max <= 64
 *   cutoff      truncation threshold as in mps_create
 *   U           host pointer, 4 x 4 complex128 row-major (not checked for unitarity)
 *   stream      cudaStream_t to run on (NULL = the legacy default stream)
 * The first call on a device looks up that device's scratch address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and each call clears what must start at
 * zero; calls that overlap on the GPU (other streams, other threads) race on
 * it and must be serialised by the caller. Synchronises `stream`.
 * Errors: MPS_ERR_ARG, MPS_ERR_TOO_LARGE (chi_max > 64), MPS_ERR_CUDA,
 * MPS_ERR_NOCONVERGE (tensors left unchanged). */
int mps_gate2_update_noalloc(double* d_gamma_l, double* d_gamma_r, const double* d_lambda_l, double* d_lambda_m,
                             const double* d_lambda_r, int* d_chi, int chi_max, double cutoff, const double* U,
                             void* stream);

/* mps_split_zgemm - C = A B for complex128 matrices in DEVICE memory,
 * column-major (A[r + k lda], B[k + n ldb], C[r + n ldc]), computed by the
 * split-precision scheme of MPS_PREC_SPLIT: each row of A and column of B is
 * scaled by a power of two and cut into `slices` signed 7-bit bf16 digits,
 * the slice products run on the tcgen05 tensor cores with exact fp32
 * accumulation, and the binary64 result is reassembled (Ozaki et al. 2012).
 * With 8 slices the result is binary64-accurate relative to |A||B|. The fp32
 * sums are exact for K <= 512; a longer K runs in 512-wide chunks whose
 * binary64 results are accumulated.
 *   M, N, K >= 1; slices 1..8
 *   stream  cudaStream_t (NULL = legacy default stream); synchronised.
 * Not a paper entry point: the building block of the split-precision update,
 * exposed for tests and reuse. Errors: MPS_ERR_ARG, MPS_ERR_TOO_LARGE,
 * MPS_ERR_NOMEM, MPS_ERR_CUDA, MPS_ERR_TIMEOUT (a bounded device wait ran out). */
int mps_split_zgemm(int M, int N, int K, const double* dA, long long lda, const double* dB, long long ldb,
                    double* dC, long long ldc, int slices, void* stream);

/* ---- Beyond binary64: double-word MPS for small bond dimensions ----------
 * The paper runs the whole simulation in MPFR multiprecision (Sec. 1; the
 * Sec. 3.2 example sets 256 bits) so that the Schmidt spectra of Eq. (2),
 * which span many orders of magnitude, keep their small values. This
 * separate handle keeps the Vidal form of Eq. (1) in double-word arithmetic
 * (a value is the unevaluated sum hi + lo of two doubles, about 106
 * significant bits) and runs every step of the Sec. 3.1 update in it:
 * theta, the one-sided Jacobi SVD, truncation, renormalisation and the
 * Lambda^-1 rewrite. Bond dimensions up to 32; one- and two-qubit gates.
 * Truncation keeps sigma_j > max(cutoff, Mw 2^-104) ||sigma||, at most
 * chi_max values, at least one (Mw: rows of the Jacobi working matrix).
 * Calls on one handle run in order on its stream; errors found on the device
 * (MPS_ERR_NOCONVERGE) are reported by the next synchronising call, and the
 * gate that failed leaves its tensors unchanged. */
typedef struct mps_dd_state* mps_dd_handle;

/* n >= 2 qubits in |0...0>; 1 <= chi_max <= 32 (MPS_ERR_TOO_LARGE above);
 * 0 <= cutoff < 1. Errors: MPS_ERR_ARG, MPS_ERR_TOO_LARGE, MPS_ERR_NOMEM,
 * MPS_ERR_CUDA. */
int mps_dd_create(int n, int chi_max, double cutoff, mps_dd_handle* out);
int mps_dd_destroy(mps_dd_handle h);
/* Back to |0...0>, counters cleared. */
int mps_dd_reset(mps_dd_handle h);
/* Runs the handle's work on `stream` (cudaStream_t; NULL = legacy default). */
int mps_dd_set_stream(mps_dd_handle h, void* stream);
/* Sweep limit of one SVD, 1..60 (default 60). */
int mps_dd_set_limits(mps_dd_handle h, int max_sweeps);

/* mps_dd_apply_layer - n_gates gates on disjoint qubits, k = 1 (U(2) on
 * sites[g]) or k = 2 (U(4) on sites[g], sites[g]+1), Sec. 3.1. U_hi holds
 * the gates as complex128 2^k x 2^k row-major matrices, gate after gate (host
 * pointer); U_lo (host, same layout, may be NULL) holds low parts, each gate
 * entry being hi + lo exactly. Both are copied before the call returns; the
 * update runs asynchronously. Errors: MPS_ERR_ARG (k, range, overlap),
 * MPS_ERR_CUDA. */
int mps_dd_apply_layer(mps_dd_handle h, int k, int n_gates, const int* sites, const double* U_hi,
                       const double* U_lo);
/* The same with the layer already in device memory: d_sites (n_gates ints),
 * d_U_hi / d_U_lo (as above, d_U_lo may be NULL) are read by the kernels when
 * they run, so they must stay valid until the handle's stream has passed
 * them. `sites` (host copy of d_sites) is used to check the layer. */
int mps_dd_apply_layer_device(mps_dd_handle h, int k, int n_gates, const int* sites, const int* d_sites,
                              const double* d_U_hi, const double* d_U_lo);
/* Waits for the handle's stream; reports a deferred device error, clearing it. */
int mps_dd_sync(mps_dd_handle h);
/* n+1 bond dimensions (chi[0] = chi[n] = 1). Synchronises. */
int mps_dd_bond_dims(mps_dd_handle h, int* chi);
/* Lambda_bond (Eq. 2), descending: hi and lo parts (either may be NULL),
 * *len values (at most chi_max). Synchronises. */
int mps_dd_get_schmidt(mps_dd_handle h, int bond, double* hi, double* lo, int* len);
/* <b|psi> of Eq. (1) for `count` bit strings (bits[count][n], one byte per
 * qubit, 0/1): out[count][4] = (re hi, re lo, im hi, im lo). Synchronises.
 * Errors: MPS_ERR_ARG, MPS_ERR_NOMEM, MPS_ERR_CUDA. */
int mps_dd_amplitudes(mps_dd_handle h, int count, const unsigned char* bits, double* out);
/* Two-site updates issued since create/reset, Jacobi sweeps they ran, and
 * the binary64 operations the theta and Jacobi kernels executed (counted on
 * the device). Synchronises. Any output may be NULL. */
int mps_dd_stats(mps_dd_handle h, long long* updates, long long* sweeps, double* flops);

/* ---- Hermitian matrices: the library's second workload --------------------
 * Sec. 2 lists the diagonalisation of a Hermitian matrix among the matrix
 * library's functions, and its NMR example (Sec. 2.1) builds a thermal state
 * with exp_H(-(h / k_B T) H), normalises it by its trace, tilts a spin with a
 * pulse, records <X> of that spin under H at intervals dt, zero-pads the
 * record and takes the modulus of its DFT. These calls do each step on the
 * GPU for `count` independent problems at once. Matrices are D x D
 * complex128, row-major, one after another in DEVICE memory; 1 <= D <= 64
 * (MPS_ERR_TOO_LARGE above). Every call synchronises `stream` (cudaStream_t,
 * NULL = legacy default) and allocates its scratch with cudaMalloc.
 * Errors: MPS_ERR_ARG, MPS_ERR_TOO_LARGE, MPS_ERR_NOMEM, MPS_ERR_CUDA,
 * MPS_ERR_NOCONVERGE (a Jacobi sweep limit of 60 was hit). */

/* Eigenvalues in ascending order d_w[count][D] and eigenvectors
 * d_V[count][D][D] (complex128, column k of problem b is the eigenvector of
 * d_w[b][k]) of Hermitian d_H (only the Hermitian part is meaningful: the
 * diagonal's imaginary parts are ignored). Cyclic two-sided Jacobi; a pair is
 * rotated while |h_pq| > D 2^-53 ||H||_F. */
int mps_heev_batched(int count, int D, const double* d_H, double* d_w, double* d_V, void* stream);

/* kind 0: d_out = exp(a H) for the complex scalar a = a_re + i a_im (exp_H of
 * Sec. 2.1; a = -i t gives the propagator exp(-i H t)).
 * kind 1: d_out = exp(-beta H) / Tr exp(-beta H) with beta = a_re (the
 * thermal state), computed in H's eigenbasis with the weights shifted so that
 * the largest is 1.
 * kind 2: d_out = exp(-beta H) / Tr exp(-beta H) - I / D (beta = a_re), the
 * deviation from the infinite-temperature state, with the weights formed by
 * expm1 so that it keeps full relative accuracy when beta ||H|| is small (at
 * 300 K and Hz-scale H the thermal state's entries differ from 1/D only in
 * the 10th or later digit, and the record of a traceless observable depends
 * on that difference alone). */
int mps_hermitian_function_batched(int count, int D, const double* d_H, int kind, double a_re, double a_im,
                                   double* d_out, void* stream);

/* Free-induction decay: with rho' = P rho P^H (d_P NULL: rho' = rho),
 * d_signal[b][m] = Tr(exp(-i H t_m) rho' exp(i H t_m) O), t_m = m dt,
 * m = 0..N-1 (complex128), evaluated in H's eigenbasis as
 * sum_jk rho~_jk O~_kj exp(-i (lambda_j - lambda_k) t_m) with each phase
 * computed directly from t_m. count <= 65535. */
int mps_fid_batched(int count, int D, const double* d_rho, const double* d_H, const double* d_O, const double* d_P,
                    double dt, int N, double* d_signal, void* stream);

/* Statistics of the last Jacobi diagonalisation run on the calling thread
 * (by any of the three calls above): the largest sweep count over the batch
 * and the total number of 2 x 2 rotations applied (each rotation updates two
 * rows of H and two columns of H and of V: 60 D + 25 binary64 operations). */
int mps_hermitian_last_stats(long long* max_sweeps, long long* rotations);

/* |DFT| of each of `count` complex128 records of n_in values zero-padded to
 * n_out (a power of two, 2 <= n_out <= 2^26, n_out >= n_in):
 * d_abs[b][f] = |sum_m x_m exp(-2 pi i f m / n_out)|, by a radix-2 FFT.
 * count <= 65535. */
int mps_dft_abs_batched(int count, int n_in, const double* d_x, int n_out, double* d_abs, void* stream);

/* Message describing the last error returned on the calling thread. */
const char* mps_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PAPER_1111_3124_GB300_MPS_H */
