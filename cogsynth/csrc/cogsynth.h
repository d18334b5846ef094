/*
 * cogsynth.h -- CUDA twin of cogsynth.scene (seeded synthetic surveillance
 * video).  Input generation only: it holds none of the background-
 * subtraction method's arithmetic.  Renders frames bit-identical to the
 * numpy renderer from the same static scene maps and per-frame descriptors
 * (both built by cogsynth.scene on the host).
 */
#ifndef COGSYNTH_H
#define COGSYNTH_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define COGSYNTH_MAX_OBJ 16

typedef struct {
    int32_t width, height, n_blobs, pad;
    int32_t sway_x0, sway_y0, sway_x1, sway_y1;
    const uint8_t *bg;          /* device [P][3] background texture          */
    const uint8_t *sig16;       /* device [P] noise sigma in 1/16 levels      */
    const int16_t *blob_id;     /* device [P] disc index or -1                */
    const int16_t *blob_delta;  /* device [n_blobs][3] second-mode offset     */
} cogsynth_scene;

typedef struct {
    uint64_t noise_base;        /* per-frame hash key                          */
    int32_t offset, sway, n_obj, pad;
    uint32_t modes[8];          /* bit b: disc b shows its second mode         */
    int32_t obj[COGSYNTH_MAX_OBJ][8]; /* kind(0 rect,1 ellipse), a0,b0,a1,b1, r,g,b */
} cogsynth_frame;

/* Renders n frames: out_dev[n][P][3]; gt_dev[n][P] (255 inside an object)
 * unless NULL.  frames_dev: device array of n descriptors.  stream: a
 * cudaStream_t or NULL.  Returns 0 or a cudaError_t value. */
int cogsynth_render(const cogsynth_scene *sc, const cogsynth_frame *frames_dev, int32_t n,
                    uint8_t *out_dev, uint8_t *gt_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif
