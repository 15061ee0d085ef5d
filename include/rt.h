/*
 * rt.h -- C ABI of the GB300 (sm_103a) specular radio ray tracer.
 *
 * The calls follow the problem statement of "Sionna RT: Differentiable Ray
 * Tracing for Radio Propagation Modeling" (arXiv 2303.11103):
 *   load_scene          Sec. II   triangle meshes with radio materials (eps_r, sigma)
 *   set_tx / set_rx     Sec. II-A Listing 2: positions, yaw/pitch/roll, antenna patterns
 *   compute_paths       Sec. II-B heuristic: Fibonacci-lattice rays, specular bounces,
 *                                 image-method refinement, duplicate removal, LOS added
 *   cir                 Sec. II-A Listing 3: path coefficients a_i and delays tau_i
 *   freq_response       Sec. III-A: OFDM frequency response H(f) = sum_i a_i e^{-j2 pi f tau_i}
 *   coverage_map        Sec. II-A Listing 2, Fig. 2: path-gain map on a cell grid
 *   *_backward          Sec. I/II: gradients w.r.t. materials and transmitter pose
 *
 * Conventions (every call):
 *   - Returns RT_OK (0) or a negative RT_ERR_* code; rt_last_error() gives the
 *     message. No exception or abort crosses the ABI.
 *   - SI units: metres, seconds, hertz, siemens per metre; angles in radians.
 *   - Array pointers are DEVICE pointers owned by the caller unless the
 *     parameter name ends in _host. The library copies what it keeps.
 *   - Work is enqueued on the context's stream (rt_create / rt_set_stream);
 *     calls that return counts synchronise that stream.
 *   - Complex numbers are interleaved (re, im) float32 pairs.
 *   - A context is used by one host thread at a time.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_ERR_INVALID_ARG (-1)
#define RT_ERR_CUDA (-2)
#define RT_ERR_OOM (-3)
#define RT_ERR_CAPACITY (-4)
#define RT_ERR_TIMEOUT (-5)
#define RT_ERR_NOT_READY (-6)

/* path-type flags of rt_compute_paths / rt_cir (Listing 3: cir(los, reflection)) */
#define RT_LOS 1u
#define RT_REFLECTION 2u
#define RT_RECORD_RAYS 0x100u /* keep per-ray hit lists (debug / parity) */

/* antenna pattern kinds (Sec. II-A: predefined patterns, single or dual polarized) */
#define RT_ANT_ISO 0     /* isotropic, field amplitude 1 */
#define RT_ANT_DIPOLE 1  /* short dipole, amplitude sqrt(1.5) sin(theta) */
#define RT_ANT_TR38901 2 /* 3GPP TR 38.901 Table 7.3-1 element, 8 dBi */

typedef struct rt_ctx rt_ctx;

/* One antenna: pattern kind and per-port polarization slant angle (0 = V,
 * pi/2 = H, +-pi/4 = cross). n_ports is 1 or 2. */
typedef struct rt_antenna {
    int32_t kind;
    int32_t n_ports;
    float slant[2];
} rt_antenna;

/* Horizontal coverage grid: cells [x0 + i*cell, x0 + (i+1)*cell) x
 * [y0 + j*cell, ...), i < nx, j < ny, on the plane z = height. */
typedef struct rt_grid {
    float x0, y0, cell, height;
    int32_t nx, ny;
} rt_grid;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream). */
int rt_create(rt_ctx** ctx, int device, void* cuda_stream);
/* Free every device buffer the context owns. Safe on NULL. */
int rt_destroy(rt_ctx* ctx);
int rt_set_stream(rt_ctx* ctx, void* cuda_stream);
/* Copy the last error message (NUL-terminated, truncated to len). */
int rt_last_error(const rt_ctx* ctx, char* buf, size_t len);
/* Carrier frequency (default 3.5e9 Hz). */
int rt_set_frequency(rt_ctx* ctx, double fc);

/*
 * Sec. II: scene = triangle meshes, each triangle with a radio material.
 * verts [n_tris*9] float32 (v0, v1, v2 of each triangle), mat_id [n_tris]
 * int32 in [0, n_mat), mat_params [n_mat*2] float32 (eps_r, sigma).
 * Builds the LBVH on the GPU. Surfaces are two-sided. n_tris may be 0
 * (every ray misses). Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_load_scene(rt_ctx* ctx, const float* verts, int64_t n_tris, const int32_t* mat_id,
                  const float* mat_params, int32_t n_mat);
/*
 * Hierarchy built over the Morton-sorted triangles by rt_load_scene (not in
 * the paper, which leaves intersection to Mitsuba 3): RT_BVH_KARRAS = radix
 * tree from the longest common prefixes of the codes (Karras 2012);
 * RT_BVH_PLOC (default) = agglomerative clustering of Morton-order
 * neighbours by merged surface area (Meister & Bittner 2018), a lower-cost
 * tree for the same leaves. Both give the same intersections (every query's
 * closest hit is independent of the tree). Takes effect at the next
 * rt_load_scene. Errors: RT_ERR_INVALID_ARG for another value.
 */
#define RT_BVH_KARRAS 0
#define RT_BVH_PLOC 1
int rt_set_bvh_builder(rt_ctx* ctx, int32_t builder);
/*
 * Node layout the traversal uses (not in the paper): width 2 (default) =
 * the binary nodes; width 8 = the binary hierarchy collapsed into nodes of
 * up to 8 children, whose boxes are stored plane by plane so that a ray
 * reads each child's near and far planes by its direction octant, visiting
 * children near to far. Both give the same intersections. On the
 * 4802-triangle city the binary layout is the faster one (fewer box tests
 * per query). Takes effect at the next rt_load_scene. Errors:
 * RT_ERR_INVALID_ARG for another width.
 */
int rt_set_bvh_width(rt_ctx* ctx, int32_t width);
/*
 * The binary hierarchy of the last rt_load_scene, for inspection (not in the
 * paper; tests and measurement read it): node k = 16 float32 (HOST out,
 * nodes [cap*16]): child 0 box (lo xyz, hi xyz), child 1 box (lo xyz, hi
 * xyz), then the two child references as int32 bit patterns (>= 0:
 * internal node, < 0: leaf ~j, j the leaf's position in Morton order), then
 * two unused words. Node 0 is the root; every child has a larger index
 * than its parent. *n_nodes receives the node count (0 when the scene has
 * fewer than two triangles in the hierarchy); with nodes null or cap too
 * small only the count is written. The large triangles tested directly by
 * every query are not in the hierarchy. Synchronises the context's stream.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA.
 */
int rt_get_bvh(rt_ctx* ctx, float* nodes, int64_t cap, int64_t* n_nodes);

/*
 * Duplicate removal of the SBR candidate keys in rt_compute_paths (Sec. II-B:
 * every distinct interaction sequence is refined once): RT_DEDUP_HASH
 * (default) = open-addressing hash table of the keys, then a sort of the
 * distinct keys only; RT_DEDUP_SORT = sort of all keys, then removal of
 * equal neighbours. Both give the same candidates in the same (key) order
 * with the same witness rays (the smallest producing ray). Keys that
 * fill all 64 bits, and more than 2^28 appended keys (a table above 6 GB),
 * always take RT_DEDUP_SORT. Errors: RT_ERR_INVALID_ARG for another value.
 */
#define RT_DEDUP_HASH 0
#define RT_DEDUP_SORT 1
int rt_set_dedup(rt_ctx* ctx, int32_t mode);

/* Replace the material table (same n_mat as the scene). */
int rt_set_materials(rt_ctx* ctx, const float* mat_params, int32_t n_mat);

/*
 * Sec. II-A (Listing 2): transmitters. pos [n*3], ypr [n*3] (yaw, pitch,
 * roll; 3GPP TR 38.901 Sec. 7.1 rotation Rz(yaw) Ry(pitch) Rx(roll)),
 * pattern pat (host struct, shared by all transmitters). With the same n
 * and port count as before this is a pose update: the stored paths and
 * receiver sets are kept and rt_cir / rt_cir_backward evaluate the same
 * triangle sequences at the new pose (paths frozen, as gradients assume);
 * otherwise they are dropped.
 */
int rt_set_tx(rt_ctx* ctx, const float* pos, const float* ypr, int32_t n, const rt_antenna* pat);
/*
 * Receivers, as rt_set_tx. rx_set_offsets_host (HOST, may be NULL): CSR of
 * n_tx+1 int32 giving each transmitter its own receiver range [off[t],
 * off[t+1]) of this array (uneven receiver sets); NULL = every transmitter
 * with every receiver. Must be called after rt_set_tx when sets are given.
 * The (tx, rx) pairs are numbered: without sets t*m + r; with sets the
 * receiver index itself.
 */
int rt_set_rx(rt_ctx* ctx, const float* pos, const float* ypr, int32_t m, const rt_antenna* pat,
              const int32_t* rx_set_offsets_host);

/*
 * Sec. II-B: specular paths of every (tx, rx) pair. For each transmitter,
 * num_rays rays leave along a Fibonacci lattice on the sphere (global
 * frame) and bounce specularly up to max_depth times; every prefix of a
 * ray's triangle list is a candidate; duplicates are removed; the image
 * method keeps the candidates that reach each receiver exactly and
 * unoccluded; the LOS path is added if flags has RT_LOS. max_depth = number
 * of reflections (0 = LOS only). The path store (owned by the context)
 * lists the paths of each pair in canonical order (depth, triangle ids).
 * num_paths_out (HOST) receives the path count. Synchronises the stream.
 * Errors: RT_ERR_INVALID_ARG (no scene / devices, max_depth > 6, key width
 * over 64 bits), RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_compute_paths(rt_ctx* ctx, int32_t max_depth, int64_t num_rays, uint32_t flags,
                     int64_t* num_paths_out);
/* Sec. II-B: the launch directions the tracer shoots, rays [first,
 * first+n) of a lattice of num_rays: dirs [n*3] float32 (FP64 lattice
 * formula rounded once to FP32). */
int rt_ray_directions(rt_ctx* ctx, int64_t num_rays, int64_t first, int64_t n, float* dirs);
/* Number of (tx, rx) pairs of the current device configuration (HOST out). */
int rt_num_pairs(const rt_ctx* ctx, int64_t* n_pairs_out);
/*
 * Copy the path store. Any pointer may be NULL. offsets [n_pairs+1] int64
 * (CSR over pairs), seq [P*max_depth] int32 triangle ids (-1 padded),
 * points [P*max_depth*3] float32 reflection points, depth [P] int32,
 * length [P] float64 (path length accumulated in FP64).
 */
int rt_get_paths(rt_ctx* ctx, int64_t* offsets, int32_t* seq, float* points, int32_t* depth,
                 double* length);
/*
 * Debug / parity: the de-duplicated candidate list of the last
 * rt_compute_paths. n_out (HOST) = count U (always written); tx [U],
 * depth [U], seq [U*max_depth], witness_ray [U] (the smallest lattice index
 * of the rays that produced the candidate, -1 for LOS). Any device pointer
 * may be NULL.
 */
int rt_get_candidates(rt_ctx* ctx, int64_t* n_out, int32_t* tx, int32_t* depth, int32_t* seq,
                      int64_t* witness_ray);
/* Debug / parity (flag RT_RECORD_RAYS): hits [n_tx*num_rays*max_depth]
 * int32 triangle ids per ray and bounce, -1 after a miss. */
int rt_get_ray_hits(rt_ctx* ctx, int32_t* hits);

/*
 * Listing 3 (paths.cir): channel coefficients and delays of every stored
 * path. a [P*nrp*ntp] complex (nrp/ntp = rx/tx ports), a = lambda/(4 pi r)
 * exp(-j 2 pi frac(r/lambda)) F_rx . (Fresnel chain) . F_tx, tau [P] = r/c0
 * (absolute delay). Paths excluded by flags (RT_LOS: depth 0,
 * RT_REFLECTION: depth >= 1) get a = 0.
 */
int rt_cir(rt_ctx* ctx, uint32_t flags, float* a, float* tau);
/*
 * Path gain of every (tx, rx) pair from rt_cir's a [P*nrp*ntp]: out
 * [n_pairs*2] = (1 if the pair has a path else 0, 10 log10(sum over paths
 * and port pairs of |a|^2), or floor_db without paths). The incoherent
 * received power the paper's transmitter-orientation example maximises
 * (Sec. III-B) and the label of the path-gain surrogate.
 */
int rt_pair_gain(rt_ctx* ctx, const float* a, float floor_db, float* out);
/*
 * Sec. II-A (Listing 3, paths.apply_doppler): time evolution of the channel
 * coefficients of the stored paths from the velocities of the transmitters
 * and receivers. Path i leaves its transmitter in the unit direction k_t and
 * reaches its receiver in the unit direction k_r (image method at the
 * current positions); its Doppler shift is f_D = (v_tx . k_t - v_rx . k_r) /
 * lambda, and a_t[i][p][q][n] = a[i][p][q] exp(j 2 pi f_D n / fs) for
 * n = 0..n_steps-1. The delays do not change.
 * a [P*nrp*ntp] complex (float re, im; as from rt_cir), tx_vel [n_tx*3]
 * m/s, rx_vel [n_rx*3] m/s or NULL (receivers at rest), a_t
 * [P*nrp*ntp*n_steps] complex out; all device pointers. Errors:
 * RT_ERR_INVALID_ARG for n_steps < 1, fs <= 0 or a null pointer.
 */
int rt_apply_doppler(rt_ctx* ctx, const float* a, const float* tx_vel, const float* rx_vel, double fs,
                     int32_t n_steps, float* a_t);
/*
 * Sec. II (antenna arrays modelled synthetically after the ray tracing):
 * the paths are traced between the array centres, and every element pair
 * gets the plane-wave phase of its offsets. Element m of the transmit array
 * sits at r_m, element n of the receive array at s_n, in the devices' own
 * frames (metres; rotated by the devices' yaw/pitch/roll as the patterns
 * are). With k_t / k_r the unit departure / arrival directions of path i,
 * a_el[i][n*nrp + p][m*ntp + q] = a[i][p][q] exp(j 2 pi (k_t . R_tx r_m -
 * k_r . R_rx s_n) / lambda): element-major, port-minor indices.
 * a [P*nrp*ntp] complex (as from rt_cir), tx_elements [n_tx_el*3],
 * rx_elements [n_rx_el*3] (n = 0 with NULL: one element at the centre),
 * a_el [P*n_rx_el*nrp*n_tx_el*ntp] complex out; device pointers. Errors:
 * RT_ERR_INVALID_ARG for a negative count or a null pointer.
 */
int rt_apply_array(rt_ctx* ctx, const float* a, const float* tx_elements, int32_t n_tx_el, const float* rx_elements,
                   int32_t n_rx_el, float* a_el);
/*
 * Sec. II-B (first-order diffraction; the equations are a reading, the paper
 * leaves them to the documentation): diffracted paths tx -> edge -> rx of
 * every (tx, rx) pair of the context, kept beside the specular paths.
 * Wedges are the scene edges shared by two triangles whose planes differ,
 * matched on the exact input vertex coordinates; the solid is the smaller
 * sector between the faces (convex edges). A path touches its edge where
 * the incidence and diffraction angles with the edge agree (Keller's law),
 * strictly inside the edge, with both devices outside the solid and both
 * segments free of occluders. num_paths (HOST) receives their count.
 * Errors: RT_ERR_INVALID_ARG without scene or devices, RT_ERR_NOT_READY
 * while capturing a graph.
 */
int rt_compute_diffraction(rt_ctx* ctx, int64_t* num_paths);
/* The diffracted paths, ordered by (pair, wedge): offsets [n_pairs+1] int64
 * (CSR over pairs), wedge [P] int32 (index into rt_get_wedges), points
 * [P*3] float32 diffraction points; device pointers, any may be NULL. */
int rt_get_diffraction(rt_ctx* ctx, int64_t* offsets, int32_t* wedge, float* points);
/*
 * Channel coefficients of the diffracted paths by the uniform theory of
 * diffraction for perfectly conducting wedges (Kouyoumjian-Pathak):
 * a = lambda/(4 pi) exp(-j k (s' + s)) / sqrt(s s' (s' + s))
 *     F_rx(-k_d) . [-D_s b0 b0' - D_h p p'] . F_tx(k_i),
 * with the soft / hard coefficients D_s, D_h, the incident and diffracted
 * ray-fixed bases (b0', p') and (b0, p), and the transition function
 * evaluated in FP64; path length and carrier phase in FP64. a [P*nrp*ntp]
 * complex (float re, im), tau [P] seconds; device pointers.
 */
int rt_diffraction_cir(rt_ctx* ctx, float* a, float* tau);
/*
 * Sec. II-A (Listing 2: coverage_map(..., diffraction=True)): the
 * first-order diffracted part of a coverage map. For every transmitter and
 * every cell, the diffracted paths to the cell centre at g->height (found
 * and weighted as in rt_compute_diffraction / rt_diffraction_cir, receiver
 * antenna port 0 unrotated, transmit port tx_port) and the incoherent sum
 * of their |a|^2, the path gain the specular map estimates per cell.
 * gain [n_tx*ny*nx] float32 (device) is overwritten; add it to the
 * rt_coverage_map gain for the map with diffraction. Errors:
 * RT_ERR_INVALID_ARG for a bad grid or port or without scene and devices,
 * RT_ERR_NOT_READY while capturing a graph.
 */
int rt_coverage_map_diffraction(rt_ctx* ctx, const rt_grid* g, int32_t tx_port, float* gain);
/*
 * Sec. II-B (diffuse reflections, i.e. scattering; the model is a reading,
 * the paper leaves it to the documentation): scattering coefficients S
 * [n_mat] float32 (device, 0..1; a value <= 0 scatters nothing) of the
 * scene's materials; all zero (no scattering) until set, and reset by
 * rt_load_scene. The values stay on the device and are not checked: S > 1
 * re-radiates more power than arrives, which is outside the model, and a
 * material with S <= 0 gets a zero gradient from rt_scattering_gain_vjp, so
 * an optimiser stepping S must keep it in (0, 1] itself (clamp it, or
 * optimise an unconstrained u with S = sigmoid(u)). Errors:
 * RT_ERR_INVALID_ARG for another material count.
 */
int rt_set_scattering(rt_ctx* ctx, const float* coeff, int32_t n_mat);
/*
 * Sec. II (the radio materials carry a scattering pattern): pattern of each
 * material for rt_scattering_gain. alpha_r [n_mat] int32 (HOST, read during
 * the call): -1 the Lambertian pattern cos(theta_s)/pi (the default until
 * set, and after rt_load_scene); 0..RT_MAX_ALPHA_R the directive pattern of
 * the effective-roughness model, a lobe ((1 + k_r . k_s)/2)^alpha_r around
 * the specular direction k_r, normalised over the hemisphere on the
 * incident side so that it re-radiates the same power S^2. Errors:
 * RT_ERR_INVALID_ARG for another material count or an exponent out of range.
 */
#define RT_MAX_ALPHA_R 64
int rt_set_scattering_pattern(rt_ctx* ctx, const int32_t* alpha_r, int32_t n_mat);
/*
 * First-order diffuse scattering by the effective-roughness model with the
 * materials' patterns (rt_set_scattering_pattern; Lambertian below): each of the num_rays Fibonacci rays of a transmitter
 * carries |F_tx,q(d)|^2 / num_rays of its power; at its first hit the
 * fraction S^2 is re-radiated with the intensity cos(theta_s)/pi towards
 * the side the ray came from, and a receiver there with an unoccluded
 * segment collects lambda^2/(4 pi r^2) |F_rx,p|^2 of it, half per port
 * (depolarised wave). gain [n_pairs*nrp*ntp] float32 (device, overwritten):
 * the incoherent scattered path gain of every pair and port pair. The
 * specular coefficients are not changed. Errors: RT_ERR_INVALID_ARG.
 */
int rt_scattering_gain(rt_ctx* ctx, int64_t num_rays, float* gain);
/*
 * Sec. II (gradients with respect to the parameters of the scattering
 * functions): vector-Jacobian product of rt_scattering_gain with respect to
 * the coefficients S. grad_gain [n_pairs*nrp*ntp] float32 (device) is
 * dL/dgain; grad_coeff [n_mat] float32 (device, overwritten) receives dL/dS.
 * The gain is quadratic in S: dL/dS_m = (2/S_m) * the sum of dL/dgain times
 * the gain carried by the rays that first hit material m (0 where S_m = 0).
 * Errors: RT_ERR_INVALID_ARG.
 */
int rt_scattering_gain_vjp(rt_ctx* ctx, int64_t num_rays, const float* grad_gain, float* grad_coeff);
/* Wedges of the current scene: n_out (HOST) = count; faces [n*2] int32 the
 * two triangles (original ids, lower first), n_ext [n] exterior angle / pi;
 * device pointers, either may be NULL. Reads back (not while capturing). */
int rt_get_wedges(rt_ctx* ctx, int64_t* n_out, int32_t* faces, float* n_ext);
/*
 * Sec. III-A: H [n_pairs*nrp*ntp*K] complex, H = sum_i a_i exp(-j 2 pi f_k tau_i)
 * over the pair's paths, from a [P*nrp*ntp] and tau [P] as returned by
 * rt_cir; freqs [K] float64 baseband offsets (Hz).
 */
int rt_freq_response(rt_ctx* ctx, const float* a, const float* tau, const double* freqs,
                     int32_t K, float* H);

/*
 * Sec. III-A: rt_freq_response over a path list the caller provides rather
 * than the context's traced paths (paths from another tracer, a saved CIR,
 * synthetic channels). offsets [n_pairs+1] int64 (device, CSR: pair r owns
 * paths offsets[r] .. offsets[r+1]-1, non-decreasing, offsets[0] = 0);
 * a [P*n_port_pairs] complex64 (device, path-major); tau [P] float32
 * (device, s); freqs [K] float64 (device, Hz baseband offsets);
 * H [n_pairs*n_port_pairs*K] complex64 (device, overwritten):
 * H[r][q][k] = sum_i a[i][q] exp(-j 2 pi f_k tau_i). n_port_pairs is 1, 2
 * or 4. Needs no scene. Errors: RT_ERR_INVALID_ARG.
 */
int rt_freq_response_paths(rt_ctx* ctx, const int64_t* offsets, int64_t n_pairs, int32_t n_port_pairs,
                           const float* a, const float* tau, const double* freqs, int32_t K, float* H);

/*
 * Sec. II-A Listing 2 / Fig. 2: coverage map of every transmitter, port
 * tx_port, on grid g, by the ray-density estimator: each of num_rays
 * Fibonacci rays carries the transmit field through up to max_depth
 * specular reflections; every segment crossing z = height at x with
 * direction d adds |F_rx(-d) . E|^2 / (num_rays |d_z|) to its cell
 * (receiver pattern: rt_set_rx's, port 0, unrotated); cell gain =
 * lambda^2/(4 pi cell^2) * sum. gain [n_tx*ny*nx] float32, hits
 * [n_tx*ny*nx] uint32 (crossings per cell); both overwritten. All
 * transmitters run in one persistent launch.
 */
int rt_coverage_map(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays,
                    int32_t tx_port, float* gain, uint32_t* hits);
/*
 * As rt_coverage_map, but traces only lattice rays [first_ray, first_ray +
 * ray_count) of the num_rays lattice of every transmitter and ADDS to gain
 * and hits (not zeroed). Summing calls over a partition of [0, num_rays)
 * gives rt_coverage_map's result up to float summation order (used to split
 * large jobs and to trace chosen subsets of rays).
 */
int rt_coverage_map_accumulate(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays,
                               int64_t first_ray, int64_t ray_count, int32_t tx_port, float* gain,
                               uint32_t* hits);

/*
 * Coverage map computed concurrently with the calls that follow it (not in
 * the paper). Same inputs, outputs and result as rt_coverage_map (up to
 * float summation order), but the map is traced on a second stream of the
 * context, with its own work counter and status word, beside later calls
 * that leave the scene, materials, frequency, transmitters, receivers and
 * ray order unchanged (rt_compute_paths with the same num_rays, rt_cir,
 * rt_freq_response and their backward calls): their small kernels and host
 * round trips then fill the GPU while the map traces.
 *   flags 0: the map starts after all work queued so far on the context's
 *     stream.
 *   flags RT_ASYNC_AFTER_TRACE: the map starts after the ray trace of the
 *     next rt_compute_paths, beside its candidate refinement and the calls
 *     after it, instead of competing with the trace for the SMs; a call
 *     that needs the map earlier starts it at that point.
 *   blocks_per_sm 0 (the default): the map runs as short-lived blocks (each
 *     warp traces one refill of 32 rays, then its block ends), so that SM
 *     slots keep freeing while it traces and kernels of the context's
 *     stream take them first when that stream has the higher priority. The
 *     second stream is created at the lowest stream priority, so give the
 *     context's stream a higher one (cudaStreamCreateWithPriority) for the
 *     calls beside the map to run alongside it instead of after it.
 *   blocks_per_sm > 0: one persistent launch with at most that many resident
 *     blocks per SM.
 * rt_join(ctx) orders the context's stream after the map; read gain and hits
 * only after it, and keep them allocated until then. rt_destroy waits for a
 * started map and drops one still waiting for a path trace. The calls that change
 * what the map reads (rt_load_scene, rt_set_materials, rt_set_frequency,
 * rt_set_tx, rt_set_rx, rt_set_tuning, another coverage map, rt_autotune, a
 * rt_compute_paths with another num_rays) join first by themselves, and so
 * does rt_set_stream to another stream. Not allowed while capturing a graph
 * (RT_ERR_NOT_READY). Errors: as rt_coverage_map, and RT_ERR_INVALID_ARG
 * for blocks_per_sm < 0 or an unknown flag.
 */
#define RT_ASYNC_AFTER_TRACE 1u
int rt_coverage_map_async(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, int32_t tx_port,
                          uint32_t flags, int32_t blocks_per_sm, float* gain, uint32_t* hits);
/* Orders the context's stream after the map of rt_coverage_map_async
 * (starting it first if it is still waiting for a path trace). */
int rt_join(rt_ctx* ctx);

/*
 * Measured issue peaks for the roofline of the tracer's kernels (the paper
 * has no counterpart; this is measurement support). Runs a register-only
 * micro-kernel on the context's device and stream, six launches of about
 * 2 ms (the first is a warm-up), and writes the best rate to *ops_per_s
 * (HOST):
 *   RT_PROBE_TRAVERSAL: the traversal's own box test (planes chosen by the
 *     ray's octant: 11 operations, 6 FMA, 4 min/max, 1 compare) and
 *     Moller-Trumbore triangle test (35 operations), n_slab box tests (a
 *     positive multiple of 8) per n_tri triangle tests, as algorithmic
 *     operations per second (the counts the bench's roofline uses); the box
 *     test is timed in both forms the traversal code has (two children per
 *     packed FMA, one box per scalar FMA; six launches each) and the faster
 *     rate is written;
 *   RT_PROBE_FFMA: FP32 fused multiply-adds, as flops per second (2 per
 *     FMA); n_slab and n_tri are ignored.
 * Synchronises the stream. Errors: RT_ERR_INVALID_ARG, RT_ERR_NOT_READY
 * while capturing a graph, RT_ERR_CUDA.
 */
#define RT_PROBE_TRAVERSAL 0
#define RT_PROBE_FFMA 1
int rt_probe_peak(rt_ctx* ctx, int32_t kind, int32_t n_slab, int32_t n_tri, double* ops_per_s);

/*
 * Allocation-free coverage map. The paper has no counterpart; it exists for
 * callers that must not allocate device memory at call time: hosts whose
 * device memory is owned by another allocator (a framework's caching
 * allocator can leave cudaMalloc without room, or fragment memory it
 * manages), latency-critical loops in which cudaMalloc's implicit
 * synchronisation is not acceptable, and plug-ins whose host application
 * forbids device allocations. Same inputs, outputs and result as
 * rt_coverage_map (up to float summation order), but the call allocates
 * nothing: its scratch (work counter, status word, ray order) lives in one
 * static device array of about 4.03 MB that every GPU which loads the library
 * holds until the process exits. Limits and behaviour:
 *   - num_rays <= RT_NOALLOC_MAX_RAYS (1048576) per transmitter, else
 *     RT_ERR_INVALID_ARG with a message (use rt_coverage_map for more);
 *   - the context must already hold the scene and devices (rt_load_scene,
 *     rt_set_tx, rt_set_rx allocate; call them during set-up);
 *   - every call looks up the array's device address (cudaGetSymbolAddress)
 *     with the context's device current, so the address stays right after
 *     cudaDeviceReset or under another context of the device; the first
 *     lookup on a device may load the library's GPU module, so make the
 *     first call during set-up, before any stream capture;
 *   - like rt_coverage_map it reports no traversal overflow: every scene
 *     load checks the hierarchy on the device (a tree, depth below the
 *     traversal stack), so a query cannot overflow its stack;
 *   - all calls share the one array and each call clears what must start at
 *     zero; calls whose GPU work overlaps (other streams or contexts on the
 *     same device) race on it, so serialise them.
 */
#define RT_NOALLOC_MAX_RAYS 1048576
int rt_coverage_map_noalloc(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays,
                            int32_t tx_port, float* gain, uint32_t* hits);

/*
 * Sec. III-B: VJP of rt_coverage_map with respect to the transmitters'
 * orientation. grad_gain [n_tx*ny*nx] (device) is the upstream gradient of
 * the gain map (same grid, depth, ray count and port as the forward call);
 * grad_ypr [n_tx*3] (device) receives d(sum grad_gain * gain)/d(yaw, pitch,
 * roll), overwritten. The rays are traced again; the ray geometry does not
 * depend on the orientation, so the gradient is exact for the sampled rays.
 * Not allowed while capturing a graph (it may build the ray order).
 * Errors: RT_ERR_INVALID_ARG.
 */
int rt_coverage_map_backward(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, int32_t tx_port,
                             const float* grad_gain, float* grad_ypr);

/*
 * Sec. I/II (differentiability): vector-Jacobian products through the
 * stored paths (no re-trace). grad_a [P*nrp*ntp] complex and grad_tau [P]
 * (may be NULL) are the upstream gradients of a real loss w.r.t. rt_cir's
 * outputs (PyTorch convention dL/dRe + j dL/dIm). Accumulates (+=) into
 * g_eps [n_mat], g_sigma [n_mat], g_txpos [n_tx*3], g_txypr [n_tx*3]; any
 * may be NULL.
 */
int rt_cir_backward(rt_ctx* ctx, uint32_t flags, const float* grad_a, const float* grad_tau,
                    float* g_eps, float* g_sigma, float* g_txpos, float* g_txypr);
/*
 * VJP of rt_freq_response: from grad_H [n_pairs*nrp*ntp*K] complex, writes
 * grad_a [P*nrp*ntp] complex and grad_tau [P] (overwritten).
 */
int rt_freq_response_backward(rt_ctx* ctx, const float* a, const float* tau, const double* freqs,
                              int32_t K, const float* grad_H, float* grad_a, float* grad_tau);

/*
 * Batching (not in the paper): CUDA graph of a sequence of calls.
 * rt_graph_begin starts capturing the context's work (on an internal stream
 * when the context's stream is the legacy default stream); the calls that
 * follow are recorded instead of run. Calls that read results back to the
 * host (rt_compute_paths, rt_load_scene, rt_set_rx with receiver sets,
 * rt_profile_report, a first rt_coverage_map at a new num_rays) fail with
 * RT_ERR_NOT_READY while capturing. rt_graph_end instantiates the graph;
 * rt_graph_launch replays it on the context's stream, reading the buffers
 * the recorded calls named (update their contents in place between
 * replays). One graph per context; rt_graph_begin replaces the previous.
 * A replay is refused (RT_ERR_NOT_READY) once a later call has reallocated
 * a context buffer the graph uses (a larger scene or device set, another
 * ray count): capture again.
 */
int rt_graph_begin(rt_ctx* ctx);
int rt_graph_end(rt_ctx* ctx);
int rt_graph_launch(rt_ctx* ctx);

/*
 * Autotuner (not in the paper): times rt_coverage_map on the current scene
 * and transmitters for every candidate launch configuration of the
 * persistent tracing kernels (threads per block, rays per warp refill, BVH
 * nodes staged in shared memory), keeps the fastest for this context and,
 * if cache_path is not NULL, records it there (a text line per workload
 * key) and reuses a recorded choice when the key matches. gain/hits:
 * scratch outputs of the size rt_coverage_map needs. Synchronises.
 */
int rt_autotune(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, float* gain,
                uint32_t* hits, const char* cache_path);
/* The launch configuration in use: block threads (128|256), rays per warp
 * refill (0 = automatic, else >= 32), BVH nodes staged in shared memory
 * (<= 3200, counted in 64-byte binary nodes; used by the 8-wide layout
 * only, the binary layout reads its octant copies through L1) (HOST out /
 * in). */
int rt_get_tuning(const rt_ctx* ctx, int32_t* block, int32_t* chunk, int32_t* smem_nodes);
int rt_set_tuning(rt_ctx* ctx, int32_t block, int32_t chunk, int32_t smem_nodes);

/*
 * Learned path-gain surrogate (not in the paper; Sec. I cites neural
 * path-loss prediction as related work). f(tx, rx) = MLP(Fourier features):
 * x' = 2 (x - lo)/(hi - lo) - 1 for the 6 coordinates (tx xyz, rx xyz),
 * features [sin 2 pi B x', cos 2 pi B x'] with B [n_freq x 6] ~ N(0,
 * sigma^2), n_hidden ReLU layers of `width`, a 2-wide head: (logit of "the
 * tracer finds a path", path gain in dB). Dense layers run as tcgen05 BF16
 * GEMMs with FP32 accumulation; parameters are FP32 (Adam), BF16 copies feed
 * the GEMMs. All pointers are device pointers except *_host.
 */
typedef struct rt_mlp rt_mlp;
/* n_freq % 4 == 0, width in {64, 128, 192, 256}, 1 <= n_hidden <= 16;
 * lo_host/hi_host [6]: the normalisation box of (tx xyz, rx xyz). */
int rt_mlp_create(rt_mlp** m, int device, void* cuda_stream, int32_t n_freq, int32_t width, int32_t n_hidden,
                  float sigma, uint64_t seed, const float* lo_host, const float* hi_host);
int rt_mlp_destroy(rt_mlp* m);
int rt_mlp_set_stream(rt_mlp* m, void* cuda_stream);
int rt_mlp_last_error(const rt_mlp* m, char* buf, size_t len);
/* One Adam step on a batch: x [batch*6], target [batch*2] = (1 if the
 * tracer found a path else 0, path gain dB); loss = mean over the batch of
 * BCE(logit, has_path) + has_path ((gain_pred - gain)/20 dB)^2, ADDED to
 * loss_out[0] (device; may be NULL). batch % 128 == 0. */
int rt_mlp_train_step(rt_mlp* m, const float* x, const float* target, int32_t batch, float lr, float* loss_out);
/* Free-space baseline (wavelength in m; 0, the default, = none): with it
 * the gain output is the network's residual plus the Friis gain
 * 20 log10(lambda / (4 pi d)), d = |rx - tx| (at least 1 m), in training
 * (the loss compares the residual) and inference alike. */
int rt_mlp_set_baseline(rt_mlp* m, float wavelength);
/* out [n*2] = (path logit, path gain dB) for x [n*6]. One fused persistent
 * kernel (all layers per 128-query tile, activations kept on chip) when
 * 2*n_freq and width are multiples of 64, else rt_mlp_infer_layers. */
int rt_mlp_infer(rt_mlp* m, const float* x, int64_t n, float* out);
/* The same outputs layer by layer through rt_gemm_bf16's kernel
 * (activations through device memory). */
int rt_mlp_infer_layers(rt_mlp* m, const float* x, int64_t n, float* out);
/* Parameter vector layout: per layer W [out x in] then b [out] (hidden
 * layers, then the head), then the Fourier matrix [n_freq x 6]. */
int rt_mlp_num_params(const rt_mlp* m, int64_t* n_host);
int rt_mlp_get_params(rt_mlp* m, float* dst);
int rt_mlp_set_params(rt_mlp* m, const float* src);
/*
 * Save and load a surrogate (configs of the learned part: a model trained
 * once is reused for inference). rt_mlp_save writes the shape (n_freq,
 * width, n_hidden), the normalisation box, the free-space baseline, the
 * output scaling and the parameter vector (rt_mlp_get_params layout), with
 * a 64-bit FNV-1a hash, into buf (HOST, cap bytes); *size_out (HOST)
 * receives the byte count, and buf == NULL only queries it. Synchronises
 * the model's stream. The optimiser state (Adam moments, step) is not
 * saved: training a loaded model starts it afresh. Errors:
 * RT_ERR_INVALID_ARG, RT_ERR_CAPACITY if cap is below the size.
 * rt_mlp_load creates a model on device/cuda_stream from such bytes (buf
 * HOST, size bytes); outputs equal the saved model's bit for bit. Errors:
 * RT_ERR_INVALID_ARG for a size, magic or hash mismatch; as rt_mlp_create.
 */
int rt_mlp_save(rt_mlp* m, void* buf, int64_t cap, int64_t* size_out);
int rt_mlp_load(rt_mlp** m, int device, void* cuda_stream, const void* buf, int64_t size);
/* Gradients of the last training step (before its update), parameter layout. */
int rt_mlp_get_grads(rt_mlp* m, float* dst);
/* Error bits of the GEMM kernels (1 = a bounded wait timed out) (HOST out). */
int rt_mlp_status(rt_mlp* m, uint32_t* status_host);
/* C [M x N] = act(A [M x K] B [N x K]^T + bias [N]) with BF16 A, B (row-major)
 * on tcgen05; act = ReLU if relu; C BF16 if out_bf16 else FP32; N % 8 == 0,
 * K % 8 == 0; status (device, may be NULL) receives timeout bits. */
int rt_gemm_bf16(void* cuda_stream, const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                 const float* bias, int32_t relu, int32_t out_bf16, void* C, uint32_t* status);

/*
 * Instrumentation (the paper describes none; used for measurement).
 * rt_profile(flags): bit 0 (RT_PROFILE_TIME) = CUDA-event timing of every
 * kernel the context launches (events recorded on the context's stream right
 * around each launch); bit 1 (RT_PROFILE_COUNT) = the traversal kernels
 * count BVH node / triangle records and queries (a separately compiled
 * variant; without the bit they count nothing); 0 stops both; clears earlier
 * records. rt_profile_report: synchronises and
 * writes JSON {"launches": kernel launches since the last reset,
 * "kernels": {name: [launches, total ms]}, "closest_hit": closest-hit
 * queries, "any_hit": visibility queries, "plane_segments": the coverage
 * rays' last segments tested up to the map plane (any-hit queries of the
 * coverage kernels), "nodes": BVH node records fetched (all queries),
 * "tris": triangle records fetched, "sbr_keys": candidate keys the
 * last shooting pass appended, "candidates": distinct candidates, "paths":
 * valid paths of the last rt_compute_paths}; reset != 0 zeroes the
 * counters afterwards. RT_ERR_CAPACITY if buf is too small (truncated).
 */
#define RT_PROFILE_TIME 1
#define RT_PROFILE_COUNT 2
int rt_profile(rt_ctx* ctx, int flags);
int rt_profile_report(rt_ctx* ctx, char* buf, size_t len, int reset);
/* Restrict the event timing of rt_profile to the kernels named in `names`
 * (HOST, comma-separated, e.g. "k_coverage,k_sbr"); NULL or "" times every
 * kernel again. Launch counting is unaffected. */
int rt_profile_select(rt_ctx* ctx, const char* names);

#ifdef __cplusplus
}
#endif
#endif
