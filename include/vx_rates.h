/*
 * vx_rates.h -- C ABI of the GB300 (sm_103a) pair-process rate library.
 *
 * The library evaluates, for every radial zone of every ray, the e+e- <-> nu nubar pair kernel
 * Phi_l(eps, eps') (l = 0, 1) and contracts it with the zone's partner neutrino spectra into
 * emissivities and opacities, plus their derivatives with respect to the zone state.
 *
 * Where it sits in the method. Marek et al. (arXiv:1404.1719) solve the neutrino moment equations
 * ray by ray (sec. 2.1): each ray's radial sweep is an implicit Newton-Raphson solve with an
 * explicit Jacobian, and the neutrinos' emission, absorption and scattering rates are among the
 * components that solve needs (sec. 2.1). Rays are independent (sec. 2.2), and parallelism
 * inside a ray's phase space is the paper's stated next step (sec. 4). The paper does not write
 * the rate kernels down; the kernel evaluated here is the standard electroweak pair kernel with
 * massless leptons and Fermi-Dirac blocking, under these readings:
 *   - Gauss-Legendre in cos(omega) with n_mu nodes and Gauss-Legendre on the finite electron
 *     energy interval [E-, E+] with n_e nodes;
 *   - Legendre convention R = sum_l (2l+1)/2 Phi_l P_l(cos omega);
 *   - partner spectra f(mu') = J + 3 mu' H, where J, H are the occupation moments of the
 *     moment equation of sec. 2.1;
 *   - couplings (C_V +- C_A)^2 with sin^2(theta_W) = sin2w. nu_e pairs with anti-nu_e (whose kernel
 *     is the transpose), and nu_x pairs with its own spectrum;
 *   - C = c/(2 pi hbar c)^3 is the phase-space constant of sec. 2.1 (config field `norm`).
 *   Outputs, per zone z, species s and bin i:
 *     j0   = 2 pi C sum_j w_j Phi^p_0(i,j) (1 - Jbar_j),   chi0 = 2 pi C sum_j w_j Phi^a_0(i,j) Jbar_j,
 *     j1   = 6 pi C sum_j w_j Phi^p_1(i,j) Hbar_j,         chi1 = 6 pi C sum_j w_j Phi^a_1(i,j) Hbar_j,
 *   with w_j = eps_j^2 d(eps_j), Jbar/Hbar the partner's moments, so that the source term of the
 *   occupation f(eps, mu) is (1 - f)(j0 - mu j1) - f (chi0 + mu chi1).
 *
 * Conventions for every entry point:
 *   - All arrays are dense, row-major, 64-bit IEEE doubles unless stated; "device" pointers are
 *     CUDA global memory of the current device, owned by the caller. The library never frees
 *     caller memory and never retains a caller pointer after a call returns.
 *   - eval/adjoint are asynchronous on `stream`. All argument checks happen on the host before
 *     anything is launched; a rejected call returns VX_ERR_INVALID_ARG and writes nothing.
 *   - Numeric problems found on the device (T <= 0 or non-finite, |eta_e| > 80, a non-finite
 *     result) do not trap: the zone's outputs are set to NaN and a device flag is raised, which
 *     vx_rates_check() reports as VX_ERR_NUMERIC.
 *   - A handle is not thread-safe; use one handle per host thread / stream.
 */
#ifndef VX_RATES_H
#define VX_RATES_H

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (identical to cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *vx_stream;

typedef enum {
    VX_OK = 0,
    VX_ERR_INVALID_ARG = 1, /* bad pointer, size, config or layout; nothing was launched      */
    VX_ERR_CUDA = 2,        /* a CUDA runtime call failed (message via vx_last_error())       */
    VX_ERR_OOM = 3,         /* the library could not allocate its own tables                  */
    VX_ERR_NUMERIC = 4,     /* a device-side numeric check failed (see conventions above)     */
    VX_ERR_UNSUPPORTED = 5, /* valid request outside what this build supports                 */
    VX_ERR_TIMEOUT = 6      /* reserved: a bounded device wait gave up                        */
} vx_status;

typedef enum {
    VX_PREC_FP64 = 0,  /* plain FP64 quadrature (forward only): the comparison baseline        */
    VX_PREC_MIXED = 1  /* FP32 quadrature; extra precision on the degeneracy-sensitive steps   */
} vx_precision;

typedef enum { VX_NU_E = 0, VX_NU_EBAR = 1, VX_NU_X = 2 } vx_species;

/* flags */
#define VX_USE_GRAPH 1u /* launch through a cached CUDA graph (memset + persistent kernel)      */
#define VX_AUTOTUNE 2u  /* pick launch shapes by timing them on the first batch; cached on disk
                           in the JSON file named by the environment variable VX_AUTOTUNE_CACHE
                           (default: no file)                                                   */
#define VX_QUAD_SPLIT 4u /* split discrete rule in electron energy: in zones with |eta_e| >
                            eta_fp64, where the Fermi edge of the degenerate lepton (E = mu_e
                            for eta >= 0, Ebar = -mu_e for eta < 0) lies inside (E-, E+), two
                            Gauss-Legendre panels of n_e/2 nodes meet at it; elsewhere the
                            standard n_e-node rule. It converges much faster at high
                            degeneracy. n_e must be even; mixed precision only
                            (VX_ERR_UNSUPPORTED with VX_PREC_FP64)                           */
#define VX_PRECISE 8u    /* precise mode of the mixed form, for outputs whose sums cancel: the
                            electron argument of the blocking factor is formed exactly (split
                            on a per-zone power-of-two grid) in every zone, not only where
                            |eta_e| > eta_fp64, and every projection onto l = 0, 1 over
                            cos(omega), the combination of partial projections and the spectral
                            contraction are carried in double-float (FP32 pairs). It bounds the
                            error of the l = 1 results and of the eta-tangents, whose sums
                            cancel, at about 1e-7 of their sums of absolute values (see the
                            tests for the measured bounds); it costs ~15-25 % more time. Mixed
                            precision only (VX_ERR_UNSUPPORTED with VX_PREC_FP64)              */

typedef struct {
    int n_bins;             /* N, 2..31 energy bins                                           */
    const double *eps;      /* host [N], bin centres in MeV, strictly increasing, > 0         */
    const double *weights;  /* host [N] w_i = eps_i^2 d(eps_i), or NULL: edges at geometric
                               midpoints, outer edges half a logarithmic step out              */
    int n_mu;               /* Gauss-Legendre nodes in cos(omega), 2..64                      */
    int n_e;                /* Gauss-Legendre nodes in electron energy, 2..64                 */
    int n_species;          /* S, 1..3                                                        */
    const int *species;     /* host [S] vx_species values, distinct; nu_e and anti-nu_e must
                               come together (each is the other's partner)                    */
    double sin2w;           /* sin^2(theta_W), e.g. 0.23                                      */
    double g2;              /* global kernel scale (G^2 in the kernel's units), e.g. 1.0      */
    double norm;            /* phase-space constant C of the contraction, e.g. 1.0            */
    double eta_fp64;        /* |eta_e| above which the mixed form uses its extended-precision
                               argument and l = 1 accumulation path (0 -> default 20)         */
    vx_precision prec;
    unsigned flags;
} vx_config;

typedef struct vx_rates vx_rates; /* opaque handle */

/* Validates the config, builds the quadrature tables in FP64 on the host and uploads them.
 * Must be called with the target device current; the handle is bound to that device.
 * Returns VX_ERR_INVALID_ARG (bad config), VX_ERR_OOM or VX_ERR_CUDA; *out is NULL then. */
vx_status vx_rates_create(const vx_config *cfg, vx_rates **out);

typedef struct {
    int n_rays;               /* R >= 0                                                        */
    long long n_zones;        /* Z >= 0 (zones of all rays, concatenated ray by ray)           */
    const int *ray_offsets;   /* device int32 [R+1] or NULL (one ray), as in vx_btd_solve:
                                 offsets[0] = 0, non-decreasing, offsets[R] = Z. Rays may be
                                 ragged; the rate of a zone does not depend on its ray, so the
                                 layout is only validated, on the device by the launch: offsets
                                 that are not such a partition raise the device flag
                                 (vx_rates_check: VX_ERR_NUMERIC, "invalid ray offsets") and every
                                 zone is still evaluated. A pointer that is not device memory, or
                                 R = 0 with Z > 0, is rejected on the host (VX_ERR_INVALID_ARG).
                                 The host-buffer calls below take a HOST array instead, validated
                                 on the host like the rest of their arguments.                   */
    const double *state;      /* device [Z][4]: T (MeV, > 0), eta_e = mu_e/T, Y_e, rho (g/cm^3) */
    const double *J;          /* device [Z][S][N]: 0th occupation moment of each species' own
                                 spectrum (species in config order)                             */
    const double *H;          /* device [Z][S][N]: 1st occupation moment                        */
} vx_batch;

typedef struct {
    double *j0, *chi0, *j1, *chi1; /* device [Z][S][N] each                                       */
    double *phi; /* device [Z][2 dir][2 l][N][N] or NULL: the raw kernel Phi^dir_l(i,j) of
                    coupling term I (dir 0 = production, 1 = annihilation), G2 applied; term II
                    is its transpose                                                           */
} vx_out;

/* Forward evaluation: rates of every zone into *out. */
vx_status vx_rates_eval(vx_rates *h, const vx_batch *batch, const vx_out *out, vx_stream stream);

/* Derivatives with respect to the zone state, from one pass that recomputes the Fermi-Dirac
 * factors (nothing from eval is stored). Any of the outputs may be NULL, not all:
 *   jac        device [Z][S][N][4][3]: d(j0, chi0, j1, chi1)/d(T, eta_e, Y_e); the Y_e column is 0
 *   grad_state device [Z][4]: vector-Jacobian product sum_{o,s,i} grad_out_o[z,s,i] d o/d state;
 *              needs grad_out (device [Z][S][N] per output, NULL members count as 0); the
 *              Y_e and rho entries are 0
 *   fwd        forward rates of the same pass (its phi member must be NULL)
 * Mixed precision only (VX_ERR_UNSUPPORTED for an FP64 handle). */
vx_status vx_rates_adjoint(vx_rates *h, const vx_batch *batch, const vx_out *grad_out,
                           double *jac, double *grad_state, const vx_out *fwd, vx_stream stream);

/* Derivatives with respect to the partner spectra, which the rates are contracted with
 * (sec. 2.1: emissivities and opacities from the kernel and the neutrino spectra). The rates are
 * affine in J (j0 through 1 - J, chi0 through J) and linear in H (j1, chi1), so these are exact
 * and independent of J and H; with the T / eta Jacobian of vx_rates_adjoint they are the
 * zone's blocks of the Newton matrix of an implicit transport step (sec. 2.2). One pass of the
 * forward kernel; any of the outputs may be NULL, not all:
 *   blocks  device [Z][S][4][N][N]: [z][s][0][i][j] = d j0[z][s][i] / d J[z][p(s)][j],
 *           [1] = d chi0 / d J, [2] = d j1 / d H[z][p(s)][j], [3] = d chi1 / d H, where p(s) is
 *           the index (in config order) of the partner species whose spectrum species s reads
 *           (nu_e <-> anti-nu_e, nu_x with itself)
 *   grad_J, grad_H  device [Z][S][N], both or neither: vector-Jacobian product of grad_out with
 *           the blocks, indexed by spectrum, i.e. d(sum_o <grad_out_o, o>)/d J and d/d H; needs
 *           grad_out (NULL members count as 0)
 *   fwd     forward rates of the same pass (its phi member must be NULL)
 * Invalid zone states give NaN in every output of the zone and raise the device flag. Mixed
 * precision only (VX_ERR_UNSUPPORTED for an FP64 handle). */
vx_status vx_rates_spectral(vx_rates *h, const vx_batch *batch, const vx_out *grad_out, double *grad_J,
                            double *grad_H, double *blocks, const vx_out *fwd, vx_stream stream);

/* Host-buffer forms of vx_rates_eval, vx_rates_adjoint (forward rates and Jacobian) and
 * vx_rates_spectral: the batch's ray_offsets, state, J and H, the seeds and every output are HOST
 * arrays in the layouts above (pinned memory lets the copies run asynchronously); ray offsets
 * that are not a partition of the zones are rejected with VX_ERR_INVALID_ARG. The library copies the
 * batch in chunks of zones through two staging slots of device memory it owns (640 MiB each, or
 * the MiB given by the environment variable VX_HOST_SLOT_MB; allocated on the handle's first such
 * call and kept until vx_rates_destroy), on two streams of its own,
 * so one chunk's copies overlap the next chunk's kernel. Synchronous: returns when the outputs
 * are in host memory. Output rules as for the device calls; out->phi must be NULL. Mixed
 * precision only. */
vx_status vx_rates_eval_host(vx_rates *h, const vx_batch *host_batch, const vx_out *host_out);
vx_status vx_rates_adjoint_host(vx_rates *h, const vx_batch *host_batch, double *host_jac, const vx_out *host_fwd);
vx_status vx_rates_spectral_host(vx_rates *h, const vx_batch *host_batch, const vx_out *host_grad_out,
                                 double *host_grad_J, double *host_grad_H, double *host_blocks,
                                 const vx_out *host_fwd);

/* Synchronises `stream`, reads and clears the device numeric flag: VX_OK or VX_ERR_NUMERIC. */
vx_status vx_rates_check(vx_rates *h, vx_stream stream);

/* Entries of the kernel per zone and l (N*N) and the nodes per (zone, bin pair) the quadrature
 * evaluates (n_mu * n_e); for throughput accounting. */
long long vx_rates_entries_per_zone(const vx_rates *h);

/* Releases the handle's tables, graphs and scratch; NULL is a no-op. Synchronises the device. */
void vx_rates_destroy(vx_rates *h);

/* Allocation-free forward evaluation (mixed form). The paper has no counterpart: this entry point
 * exists for callers that must not have the library allocate device memory -- for example a
 * transport code that hands all device memory to its own pool allocator before time stepping,
 * or one whose implicit time step cannot afford the device-wide synchronisation that cudaMalloc
 * and cudaFree imply. It takes the config directly (no handle) and computes the same rates as
 * vx_rates_eval on a mixed-precision handle; the caller passes inputs and outputs as there.
 *   - Scratch: one file-scope device array of 307,456 bytes (work counter, numeric flag and the
 *     bin-pair table), present on every device that loads the library until the process exits.
 *     The call performs no cudaMalloc, cudaFree or other allocation.
 *   - Limits: at most 24 energy bins and 32 cos(omega) nodes; larger configs are rejected with
 *     VX_ERR_UNSUPPORTED and a message naming the limit. prec must be VX_PREC_MIXED; flags are
 *     ignored.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.
 *   - Every call on a device shares that device's copy of the array and leaves its contents behind:
 *     each call zeroes the counter and flag and rebuilds the table on `stream`, so calls whose work
 *     overlaps on the same GPU (for example on two streams) race and must be serialised by the
 *     caller. Not thread-safe.
 *   - Device-side numeric problems show up as NaN outputs of the affected zones; there is no
 *     check call for this entry point. batch->ray_offsets, if given, must be device memory but is
 *     not read (the rates do not depend on the ray layout, and there is no flag to report it). */
vx_status vx_rates_eval_noalloc(const vx_config *cfg, const vx_batch *batch, const vx_out *out, vx_stream stream);

const char *vx_status_string(vx_status s);
/* Last error message of the calling thread (static storage, never NULL). */
const char *vx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VX_RATES_H */
