/*
 * probe_stream.h -- C ABI of the GB300 probe-streaming hot path.
 *
 * The library implements the server side of "A Distributed, Decoupled System
 * for Losslessly Streaming Dynamic Light Probes to Thin Clients" (arXiv
 * 2103.05875) for one GPU: each frame it blends traced rays into the
 * octahedral irradiance and visibility texels of every probe of a volume
 * (Section 3.2), refills the one-texel guard bands (Section 3.4, Light Probe
 * Repacking), selects the probes whose transmitted codes changed since they
 * were last sent (Section 3.4, Light Probe Change Thresholding), and packs the
 * selected interiors into the lossless-video plane layouts (Section 3.3) with
 * a delta-coded 16-bit probe index buffer (Section 3.4, Light Probe Update
 * Textures). The HEVC encode itself is not part of the library: it hands back
 * packed frames.
 *
 * Conventions for every entry point:
 *  - Errors are returned as pv_status; nothing throws across the ABI.
 *    pv_last_error() gives a human-readable message for the calling thread.
 *  - "device pointer" means memory of the volume's CUDA device; "host or
 *    device" means any pointer CUDA's unified addressing resolves (pageable
 *    host, pinned host or device).
 *  - Streams are passed as an opaque cudaStream_t (void*); NULL is the legacy
 *    default stream. Asynchronous calls only enqueue work on that stream; the
 *    caller keeps inputs alive and unmodified until the stream has passed the
 *    call.
 *  - Volumes own all of their state and output buffers. A volume may be used
 *    from one host thread at a time.
 *  - Array layouts (row-major, P = nx*ny*nz probes, R rays per probe,
 *    probe id p = x + nx*(y + ny*z), n_c / n_v interior sizes, tiles of
 *    (n+2)x(n+2) texels):
 *      radiance      [3][P][R]            operand format (R, G, B planes)
 *      dist          [P][R]               operand format
 *      dirs          [R][3]               float32 unit ray directions
 *      colour tiles  [3][P][n_c+2][n_c+2] state format
 *      vis tiles     [2][P][n_v+2][n_v+2] state format (mean d, mean d^2)
 *      last codes    colour [3][P][n_c*n_c], vis [2][P][n_v*n_v] uint16;
 *                    0xFFFF marks a probe never sent
 */
#ifndef PROBE_STREAM_H
#define PROBE_STREAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pv_status {
  PV_OK = 0,
  PV_PENDING = 1,        /* pv_poll: the ticket's tick has not completed yet */
  PV_ERR_INVALID = -1,   /* bad argument, shape or descriptor field */
  PV_ERR_OOM = -2,       /* device allocation failed or memory budget exceeded */
  PV_ERR_CUDA = -3,      /* a CUDA call or kernel launch failed */
  PV_ERR_BUSY = -4,      /* no free slot in the server right now */
  PV_ERR_TIMEOUT = -5,   /* a bounded wait gave up */
  PV_ERR_RANGE = -6,     /* a size limit was exceeded (e.g. > 65536 probes) */
  PV_ERR_UNSUPPORTED = -7 /* valid request the chosen kernel cannot serve */
} pv_status;

enum { PV_FMT_F32 = 0, PV_FMT_F16 = 1, PV_FMT_BF16 = 2 };
enum { PV_CODE_UF10 = 0, PV_CODE_UNORM10 = 1 };
enum { PV_KERNEL_AUTO = 0, PV_KERNEL_SIMT = 1, PV_KERNEL_TCGEN05 = 2 };

/* Limits checked by probe_volume_create. */
#define PV_MAX_PROBES 65536   /* probe ids must fit the 2-byte index buffer (Section 3.4) */
#define PV_MAX_RAYS 1024
#define PV_MAX_INTERIOR 16    /* n_c, n_v <= 16: at most 256 texels per tile */

/*
 * Volume descriptor. The blend (Section 3.2, after DDGI) of texel t with
 * direction n_t over rays r with directions d_r:
 *   colour:     W = max(0, n_t . d_r)
 *   visibility: W = max(0, n_t . d_r)^sharpness, applied to d and d^2
 *   m = sum_r W x_r / sum_r W;  new = h*old + (1-h)*m  (a texel whose weight
 *   sum is zero keeps its value), then one rounding to state_fmt.
 */
typedef struct pv_desc {
  int32_t nx, ny, nz;           /* probe grid; P = nx*ny*nz <= PV_MAX_PROBES */
  int32_t rays_per_probe;       /* R, 1..PV_MAX_RAYS (paper: 256, Section 4) */
  int32_t color_interior;       /* n_c (paper 8, i.e. 10x10 tiles; default 6) */
  int32_t vis_interior;         /* n_v (paper 16, i.e. 18x18 tiles; default 14) */
  float hysteresis;             /* h in [0, 1) */
  float sharpness;              /* visibility cosine exponent (> 0) */
  int32_t state_fmt;            /* PV_FMT_F32 or PV_FMT_F16 */
  int32_t operand_fmt;          /* format of radiance/dist inputs and of the contraction */
  int32_t color_code;           /* PV_CODE_UF10 (default) or PV_CODE_UNORM10 */
  int32_t color_lsb;            /* 0: 16-bit sample = code << 6 (default); 1: code in low bits */
  int32_t first_frame_no_hysteresis; /* 1: the first update uses h = 0 */
  int32_t kernel;               /* PV_KERNEL_* choice of the blend kernel */
} pv_desc;

typedef struct pv_volume pv_volume;

/* Sizes of a volume's buffers and output frames (filled by probe_volume_info). */
typedef struct pv_volume_info {
  int32_t probes, rays, color_tile, vis_tile;
  int32_t blocks_w, blocks_h;                   /* update-texture block grid: nx*ny by nz */
  int32_t color_width, color_height, color_pitch_bytes; /* per colour plane (uint16 samples) */
  int32_t vis_width, vis_height, vis_pitch_bytes;       /* per visibility plane (uint8 samples) */
  int32_t kernel;                               /* blend kernel actually used */
  int32_t state_bytes_per_texel;
  uint64_t device_bytes;                        /* device memory the volume holds */
  int32_t* error_word;                          /* device int32, non-zero once a bounded wait
                                                   of the tensor-core blend gave up; read and
                                                   cleared by probe_select_and_pack with
                                                   want_host_counts (diagnostics and tests may
                                                   set it to exercise that path) */
} pv_volume_info;

/*
 * One packed update (Sections 3.3-3.4). All pointers are device pointers owned
 * by the volume and stay valid until the next probe_select_and_pack on it.
 *  color_planes  3 planes (Y=R, U=G, V=B), each color_height rows of
 *                color_pitch_bytes; sample = 10-bit code << 6 (or << 0).
 *  vis_planes    3 planes (Y, U, V), each vis_height rows of vis_pitch_bytes;
 *                the first vis_width bytes of a row are the widened byte stream
 *                of x = blocks_w*n_v RG16F texels (x' = ceil(4x/3)); the rest
 *                of the pitch is zero.
 *  index_*       probe ids of the selected probes in slot order (ascending).
 *  delta_*       the same ids delta-encoded: d0 = id0, dk = id_k - id_(k-1).
 *  count_*_dev   device uint32 counts; count_c/count_v are host copies when
 *                requested (-1 otherwise).
 * Slot k of either texture holds its probe's interior at block
 * (k / blocks_w, k % blocks_w); unused slots are zero.
 */
typedef struct pv_frame {
  uint16_t* color_planes;
  uint8_t* vis_planes;
  uint16_t* index_c;
  uint16_t* index_v;
  uint16_t* delta_c;
  uint16_t* delta_v;
  uint32_t* count_c_dev;
  uint32_t* count_v_dev;
  int64_t count_c;
  int64_t count_v;
  uint64_t frame;                               /* number of updates so far */
} pv_frame;

/* ----------------------------------------------------------------- basics */
const char* pv_status_string(pv_status s);
/* Message of the last failed call on this host thread ("" if none). */
const char* pv_last_error(void);
/* Library version string. */
const char* pv_version(void);

/*
 * Ray directions helper for callers that generate or trace rays: a spherical
 * Fibonacci set of `rays` points rotated by a uniform random rotation
 * (Shoemake 1992) drawn from SplitMix64 keyed by (seed, volume, frame).
 * The paper leaves the direction set to DDGI; the blend takes directions as an
 * input, so any set may be passed to probe_update. out_dirs: host [rays][3].
 */
pv_status pv_ray_directions(uint64_t seed, uint64_t volume, uint64_t frame, int32_t rays,
                            float* out_dirs);

/* Device bytes probe_volume_create would allocate for desc (for admission). */
pv_status probe_volume_bytes(const pv_desc* desc, uint64_t* out_bytes);

/*
 * Create a volume on the current CUDA device: tiles zero, every probe
 * "never sent", frame counter 0. Errors: PV_ERR_INVALID (bad field),
 * PV_ERR_RANGE (limits above), PV_ERR_OOM, PV_ERR_UNSUPPORTED (kernel choice
 * not available for this shape), PV_ERR_CUDA.
 */
pv_status probe_volume_create(const pv_desc* desc, pv_volume** out);
pv_status probe_volume_destroy(pv_volume* vol);
pv_status probe_volume_info(const pv_volume* vol, pv_volume_info* out);

/*
 * Blend one frame of traced rays into the volume (Section 3.2) and refill the
 * guard bands (Section 3.4); also compares the new transmitted codes with the
 * last-transmitted ones and records which probes changed (Section 3.4).
 * radiance [3][P][R], dist [P][R] in operand_fmt; dirs [R][3] float32; all
 * device pointers. Asynchronous on `stream`; advances the frame counter.
 * Errors: PV_ERR_INVALID (NULL pointer), PV_ERR_CUDA (launch failure).
 */
pv_status probe_update(pv_volume* vol, const void* radiance, const void* dist,
                       const float* dirs, void* stream);

/*
 * The two halves of probe_update, for callers that time or schedule them
 * separately: probe_update_weights computes this frame's blend weights and
 * weight sums from dirs [R][3] (device float32) and advances the frame
 * counter (K0); probe_update_blend blends radiance and dist with those weights
 * (K1: blend, hysteresis, guard band, changed flags). probe_update(v, r, d, q, s)
 * is exactly probe_update_weights(v, q, s) followed by probe_update_blend(v, r, d, s).
 */
pv_status probe_update_weights(pv_volume* vol, const float* dirs, void* stream);
pv_status probe_update_blend(pv_volume* vol, const void* radiance, const void* dist, void* stream);

/*
 * Select the changed probes and pack them (Sections 3.3-3.4): builds the
 * index buffers, writes the colour and visibility planes, and writes the sent
 * codes to the last-transmitted textures. Asynchronous unless
 * want_host_counts != 0, in which case the call waits for the stream and
 * fills out->count_c / count_v, and returns PV_ERR_TIMEOUT if a bounded
 * wait inside the tensor-core blend kernel expired since the last such call
 * (the volume's error word is set): the frames blended since then are
 * invalid, the word is cleared on `stream` and the volume stays usable.
 * Without want_host_counts the word is not read and stays set. out: host
 * pv_frame.
 */
pv_status probe_select_and_pack(pv_volume* vol, pv_frame* out, int32_t want_host_counts,
                                void* stream);

/*
 * End-to-end variants with host buffers.
 *
 * probe_update_host copies radiance, dist and dirs (host or device, layouts
 * as above) into volume-owned device staging, then runs probe_update on
 * `stream`. The staging has two halves used in turn, filled on a copy stream
 * of the volume's own, so the upload of frame f+1 runs while frame f is
 * blended; the update on `stream` waits for its upload, and a half is refilled
 * only after the blend that read it. The host buffers must stay unchanged
 * until the work this call queued on `stream` has completed; page-locked host
 * memory makes the copies asynchronous. Inside a stream capture the copies
 * are queued on `stream` itself (mixing captured and uncaptured host updates
 * of one volume needs a synchronisation between them).
 *
 * probe_frame_download copies the last packed frame to host buffers (any may
 * be NULL to skip): color [3][color_height][color_width] uint16,
 * vis [3][vis_height][vis_width] uint8, delta_c/delta_v [P] uint16 (only the
 * first count entries written), counts[2] (colour, visibility). It
 * synchronises the stream.
 *
 * probe_frame_download_async queues the same copies and returns at once with
 * a ticket (> 0). The copies run on a second stream of the volume's, after the
 * work queued on `stream` so far, so they overlap the next frame's weights and
 * blend; the volume's next probe_select_and_pack (single or batched) waits for
 * them, since it rewrites the planes in place. delta_c / delta_v receive all P
 * entries (those past the counts are unspecified). The host buffers hold the
 * frame once probe_frame_wait(vol, ticket) has returned. Host buffers should
 * be page-locked (pageable ones make the copies synchronous). Returns
 * PV_ERR_UNSUPPORTED while `stream` is being captured.
 *
 * probe_frame_wait blocks until the download of `ticket` has landed (it may
 * also wait for later downloads of the volume); PV_ERR_INVALID for a ticket
 * the volume did not issue.
 */
pv_status probe_update_host(pv_volume* vol, const void* radiance, const void* dist,
                            const float* dirs, void* stream);
pv_status probe_frame_download(pv_volume* vol, uint16_t* color, uint8_t* vis,
                               uint16_t* delta_c, uint16_t* delta_v, uint32_t* counts,
                               void* stream);
pv_status probe_frame_download_async(pv_volume* vol, uint16_t* color, uint8_t* vis,
                                     uint16_t* delta_c, uint16_t* delta_v, uint32_t* counts,
                                     uint64_t* ticket, void* stream);
pv_status probe_frame_wait(pv_volume* vol, uint64_t ticket);

/*
 * Checkpoint / resume and test injection. Buffers are host or device, layouts
 * as above (tiles in state_fmt). import also recomputes the changed-probe
 * flags against the imported last codes, so a following
 * probe_select_and_pack selects exactly what the imported state implies.
 * Both synchronise the stream. frame: number of updates so far.
 */
pv_status probe_volume_export_state(pv_volume* vol, void* tiles_c, void* tiles_v,
                                    uint16_t* last_c, uint16_t* last_v, uint64_t* frame,
                                    void* stream);
pv_status probe_volume_import_state(pv_volume* vol, const void* tiles_c, const void* tiles_v,
                                    const uint16_t* last_c, const uint16_t* last_v,
                                    uint64_t frame, void* stream);

/*
 * Allocation-free variant of probe_update (no counterpart in the paper): for
 * callers that cannot allocate device memory -- code running where cudaMalloc
 * is unavailable or not allowed, such as a stream callback, a graph host node,
 * or a plugin confined to memory its host application owns. It runs the
 * weights kernel and the SIMT blend kernel on caller buffers; its only scratch
 * (the frame's weights and their sums) is a file-scope device array of
 * PV_STATIC_SCRATCH_BYTES per GPU, held until the process exits.
 *  desc      volume descriptor (validated as by probe_volume_create).
 *  frame     number of updates the state has seen (0 on the first call; only
 *            first_frame_no_hysteresis looks at it).
 *  radiance, dist, dirs   device inputs as for probe_update.
 *  tiles_c, tiles_v       device state, read and written in place, layouts as
 *            above (unpadded tiles).
 *  last_c, last_v         device last-transmitted codes (read only).
 *  changed_bits           device output [2][ceil(P/32)] uint32: bit p%32 of word
 *            p/32 is set when probe p's colour (first half) or visibility
 *            (second half) codes differ from the last-transmitted ones.
 * Errors: PV_ERR_INVALID (NULL or bad field), PV_ERR_RANGE when the
 * weights do not fit the scratch array: with T = n_c^2 + n_v^2 texels the
 * array holds align256(4 R T) + align256(4 T) + 256 bytes at most, i.e.
 * R <= (PV_STATIC_SCRATCH_BYTES - 256 - align256(4 T)) / (4 T) (1128 rays
 * for 6x6 / 14x14 interiors, 510 for 16x16 / 16x16), PV_ERR_CUDA.
 * Asynchronous on `stream`. The first call on a device looks up the array's
 * device address, so make it before any stream capture; the address is kept
 * for the life of the process, so resetting the device after that first call
 * is not supported. All calls share the array: calls that overlap on the GPU
 * race.
 */
#define PV_STATIC_SCRATCH_BYTES (1u << 20)
pv_status probe_update_static(const pv_desc* desc, uint64_t frame, const void* radiance, const void* dist,
                              const float* dirs, void* tiles_c, void* tiles_v, const uint16_t* last_c,
                              const uint16_t* last_v, uint32_t* changed_bits, void* stream);

/* ----------------------------------------------------------------- batches */
/*
 * Batched form: up to PV_MAX_BATCH volumes with equal tile interiors, state
 * and operand formats and colour code (probe grids and rays per probe may
 * differ), all using the tensor-core blend, updated together: the weights of
 * every volume in one launch, the blend of every volume in one persistent
 * launch over all of their work items (np probes each, one CTA per SM), and
 * the selection and packing of every volume in one launch. Results equal
 * those of the same calls made volume by volume. The batch refers to the
 * volumes; they must outlive it and be used only through it while it is in
 * use. All entry points except the two tuners are asynchronous on `stream`
 * and can be captured in a CUDA graph (kernel arguments are fixed at capture).
 *  probe_batch_create   vols[n]; probes_per_item 0 picks np from the probe
 *                       count and the SM count, otherwise np (clamped to what
 *                       fits). Errors: PV_ERR_INVALID (mixed shapes, NULL,
 *                       duplicates), PV_ERR_RANGE (n > PV_MAX_BATCH),
 *                       PV_ERR_UNSUPPORTED (a volume without the tensor-core
 *                       blend), PV_ERR_CUDA.
 *  probe_batch_update   radiance[n], dist[n], dirs[n]: device inputs of each
 *                       volume as for probe_update.
 *  probe_batch_select_and_pack   out: host array of n pv_frame (device
 *                       counts only: count_c / count_v are -1).
 *  probe_batch_tune     times the blend for candidate np (8..32) with these
 *                       inputs, `reps` launches each, and keeps the fastest;
 *                       the volumes' tiles, changed bits, frame counters and
 *                       hysteresis are restored afterwards. Synchronises the
 *                       stream; out_probes_per_item (may be NULL) gets np.
 *  probe_batch_autotune the batch's plan tuned over probes per item, ray
 *                       and weight ring depths, TMEM operand stages (F32
 *                       form) and the CTA count: a coordinate search from the
 *                       default plan, each candidate timed over `reps` blend
 *                       launches with these inputs (state restored as for
 *                       probe_batch_tune), the fastest kept. cache_path (may
 *                       be NULL: no cache) names a text file of tuned plans,
 *                       one line per key; the key holds the library build
 *                       (size and modification time of the loaded library),
 *                       the device name and SM count, the formats, interiors
 *                       and every volume's probe count and rays. A key found
 *                       there is used without timing (out->from_cache = 1);
 *                       otherwise the result is appended. The file is read and
 *                       appended without locking: concurrent tuners of one
 *                       file may both append (the last line of a key wins).
 *                       Synchronises the stream. out (may be NULL): the plan
 *                       in use afterwards and the timings. Errors:
 *                       PV_ERR_INVALID (NULL argument, cache file not
 *                       writable), PV_ERR_OOM, PV_ERR_CUDA.
 *  probe_batch_info     the batch's current np.
 */
#define PV_MAX_BATCH 16
typedef struct pv_batch pv_batch;
pv_status probe_batch_create(pv_volume* const* vols, int32_t n, int32_t probes_per_item, pv_batch** out);
pv_status probe_batch_destroy(pv_batch* batch);
pv_status probe_batch_info(const pv_batch* batch, int32_t* probes_per_item);
pv_status probe_batch_update(pv_batch* batch, const void* const* radiance, const void* const* dist,
                             const float* const* dirs, void* stream);
pv_status probe_batch_select_and_pack(pv_batch* batch, pv_frame* out, void* stream);
pv_status probe_batch_tune(pv_batch* batch, const void* const* radiance, const void* const* dist,
                           const float* const* dirs, int32_t reps, int32_t* out_probes_per_item, void* stream);
typedef struct pv_tune_result {
  int32_t probes_per_item;   /* the plan in use after the call */
  int32_t ray_stages;        /* ray tile ring depth */
  int32_t weight_stages;     /* weight tile ring depth */
  int32_t tmem_stages;       /* F32 form: TMEM operand stages (0 otherwise) */
  int32_t ctas;              /* CTAs of the blend launch */
  int32_t candidates;        /* plans timed (0 when the cache answered) */
  int32_t from_cache;        /* 1: the plan came from the cache file */
  float best_us;             /* blend time of the chosen plan per launch, as tuned */
  float default_us;          /* blend time of the default plan per launch, as tuned */
} pv_tune_result;
pv_status probe_batch_autotune(pv_batch* batch, const void* const* radiance, const void* const* dist,
                               const float* const* dirs, int32_t reps, const char* cache_path,
                               pv_tune_result* out, void* stream);

/* ----------------------------------------------------------------- server */
/*
 * Served form: a request loop for many clients, each owning one probe volume
 * (a session). A session is admitted while its volume's device bytes fit the
 * memory budget and a slot is free; otherwise it waits, and waiting sessions
 * are admitted in arrival order as closing sessions free memory and slots.
 * Admitted volumes stay resident on the device. Per tick (e.g. 60 Hz), the
 * clients that submitted rays are updated together: volumes of equal shapes
 * and formats go into batches of at most max_batch (the batched form above),
 * so every client of a tick shares the same launches. Results equal those of
 * the same client served alone.
 *  pv_server_open    open session `client` for a volume `desc` (its kernel
 *                    field is ignored: the tensor-core blend is used).
 *                    PV_OK admitted, PV_PENDING waiting, PV_ERR_OOM the volume
 *                    alone exceeds the budget, PV_ERR_INVALID id in use.
 *  pv_server_close   end a session (waits for launched ticks), then admit
 *                    waiting sessions that fit.
 *  pv_server_status  admitted: 1, 0 waiting, -1 unknown client, -2 its volume
 *                    could not be created at admission (close the session);
 *                    used bytes; number of waiting sessions (outputs may be
 *                    NULL).
 *  pv_server_volume  the admitted client's volume (owned by the server, valid
 *                    until the session closes), e.g. to export its state.
 *  pv_submit         rays of an admitted client for the next tick (device
 *                    pointers, layouts as for probe_update, kept alive and
 *                    unchanged until the ticket completes); one submission
 *                    per client per tick. PV_ERR_BUSY: not admitted yet, or
 *                    already submitted for this tick.
 *  pv_server_tick    launch this tick's work on `stream` (asynchronous).
 *  pv_poll           PV_PENDING until the ticket's tick has completed on the
 *                    device, then PV_OK and the client's packed frame (device
 *                    pointers valid until the client's next tick is launched;
 *                    count_c / count_v are -1: read count_*_dev).
 */
typedef struct pv_server_desc {
  uint64_t mem_budget_bytes;    /* device bytes the admitted volumes may hold */
  int32_t max_slots;            /* sessions admitted at once */
  int32_t max_batch;            /* volumes per batched launch, 1..PV_MAX_BATCH */
} pv_server_desc;
typedef struct pv_server pv_server;
pv_status pv_server_create(const pv_server_desc* desc, pv_server** out);
pv_status pv_server_destroy(pv_server* server);
pv_status pv_server_open(pv_server* server, int32_t client, const pv_desc* desc);
pv_status pv_server_close(pv_server* server, int32_t client);
pv_status pv_server_status(pv_server* server, int32_t client, int32_t* admitted, uint64_t* used_bytes,
                           int32_t* waiting);
pv_status pv_server_volume(pv_server* server, int32_t client, pv_volume** out);
pv_status pv_submit(pv_server* server, int32_t client, const void* radiance, const void* dist,
                    const float* dirs, uint64_t* ticket);
pv_status pv_server_tick(pv_server* server, void* stream, uint64_t* tick);
pv_status pv_poll(pv_server* server, uint64_t ticket, pv_frame* out);

/* ----------------------------------------------------------------- client */
/*
 * Client side of Sections 3.3-3.4: the permanent probe textures a client keeps
 * and the decode of each packed update into them (the GPU half of the client's
 * repacking step; the video decode that would produce the planes is not part
 * of this library).
 *  pv_client_create   textures for volumes described by `desc` (the same
 *                     description as the server volume's), zeroed:
 *                     colour [3][P][(n_c+2)^2] float32, the exact values of
 *                     the transmitted codes (UF10, or UNORM10 code/1023);
 *                     visibility [2][P][(n_v+2)^2] binary16 bits (R, G), the
 *                     transmitted RG16F texels. Each tile holds the interior
 *                     and its octahedral guard band.
 *  pv_client_apply    apply one frame (asynchronous on `stream`): probe ids
 *                     from the delta-coded index buffers (delta_c/delta_v,
 *                     16-byte aligned device buffers of at least
 *                     count entries), the interiors of slots 0..count-1 from
 *                     the planes, written into the tiles of those probes,
 *                     whose guard bands are rebuilt. Reads only color_planes,
 *                     vis_planes, delta_*, count_*_dev of the frame (device
 *                     pointers laid out as probe_volume_info gives for
 *                     `desc`). Counts above P are taken as P and probe ids
 *                     at or above P are skipped. Probes not in the frame
 *                     keep their tiles.
 *  pv_client_textures device pointers of the textures (owned by the client).
 * Errors: PV_ERR_INVALID (NULL frame pointer; deltas not 16-byte aligned,
 * visibility planes not 4-byte, colour planes not 2-byte, counts not 4-byte
 * aligned; bad desc),
 * PV_ERR_RANGE / PV_ERR_OOM as probe_volume_create, PV_ERR_CUDA.
 */
typedef struct pv_client pv_client;
pv_status pv_client_create(const pv_desc* desc, pv_client** out);
pv_status pv_client_destroy(pv_client* client);
pv_status pv_client_apply(pv_client* client, const pv_frame* frame, void* stream);
pv_status pv_client_textures(const pv_client* client, float** color, uint16_t** vis);

/* ------------------------------------------------------------------ views */
/*
 * Shared-volume multi-client selection (Section 3.4: one last-transmitted
 * texture pair per client): one probe_update of a volume serves any number of
 * views, each a client's own selection and packing against what that client
 * has received.
 *  pv_view_create            a view of `vol`: its own last-transmitted codes
 *                            (nothing sent yet: its first select sends every
 *                            probe), change masks, select state and frame
 *                            buffers (about the volume's frame bytes plus its
 *                            last-code bytes). The view borrows the volume:
 *                            destroy views before their volume.
 *  pv_view_select_and_pack   as probe_select_and_pack, against the view's own
 *                            last codes: compares the volume's current codes
 *                            (those of its last update) with them, then
 *                            selects, packs into the view's frame buffers and
 *                            records what it sent. A second select without a
 *                            new update of the volume selects nothing. The
 *                            volume's own probe_select_and_pack is a separate
 *                            client and is not affected. out: host pv_frame
 *                            whose device pointers belong to the view.
 * Errors: PV_ERR_INVALID (NULL arguments), PV_ERR_OOM, PV_ERR_CUDA.
 */
typedef struct pv_view pv_view;
/*
 * Per-client selection knobs (Section 3.4; all off by default):
 *  active       device [P] bytes, nonzero for an active probe (one that may
 *               shade the client's scene); inactive probes are never sent.
 *               NULL: every probe active. Borrowed: must stay valid while
 *               the view selects.
 *  budget       at most this many probes per texture and frame (0: no
 *               limit), the first changed active probes in cyclic probe order
 *               from a per-texture cursor that then moves one past the last
 *               probe sent; probes left out stay changed and go out later.
 *  threshold_c  a probe's colour counts as changed when some texel's 10-bit
 *               code moved by more than this many code values (0: the
 *               texel-for-texel rule). Never-sent probes always count.
 *  threshold_v  the same for visibility, in binary16 ulps.
 * pv_view_set_options: PV_ERR_INVALID for negative values.
 */
typedef struct pv_view_opts {
  const uint8_t* active;
  int32_t budget;
  int32_t threshold_c;
  int32_t threshold_v;
} pv_view_opts;
pv_status pv_view_create(pv_volume* vol, pv_view** out);
pv_status pv_view_set_options(pv_view* view, const pv_view_opts* opts);
pv_status pv_view_destroy(pv_view* view);
pv_status pv_view_select_and_pack(pv_view* view, pv_frame* out, int32_t want_host_counts, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PROBE_STREAM_H */
