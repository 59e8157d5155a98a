/*
 * Parameter blocks shared by the host runtime and the kernels it compiles at
 * run time.  The same text is compiled into the host library and prepended to
 * the run-time kernel source, so both sides see one layout.
 */
#ifndef SF_KERNEL_ABI_H
#define SF_KERNEL_ABI_H

#define SF_MAX_SRC 8   /* inputs of the fused kernel: the cube and x-filtered cubes */
#define SF_MAX_NZF 4   /* spectral filters per input in the fused kernel */
#define SF_MAX_XOUT 4  /* outputs of one x-pass launch */

/* 16-bit storage types of the cube and the x-filtered scratch cubes */
struct sf_f16 { unsigned short b; };   /* IEEE binary16 */
struct sf_bf16 { unsigned short b; };  /* bfloat16 */

/* x pass: dst[k][x][y][z] = sum_o g_k[|o|] src[x+o][y][z]; lanes run over the
 * y-z plane in groups of V elements. */
struct sf_xargs {
    const void *src;
    void *dst[SF_MAX_XOUT];
    long long nx;
    long long plane;   /* ny * nz */
    long long lanes;   /* plane / V */
    long long xseg;    /* x positions per grid row */
    long long xoff;    /* first output plane of grid row 0 */
    long long nz;      /* input row length */
    long long ozs;     /* output row stride: nz, or nz padded to a 16-byte multiple (then V = 1) */
};

/* x pass of many cubes in one launch: blocks [block0, next block0) of the
 * grid take the lanes of one cube, V elements per lane. */
struct sf_xcube {
    const void *src;
    void *dst[SF_MAX_XOUT];
    long long nx;
    long long x0, x1;  /* output planes [x0, x1) (the whole cube: 0, nx) */
    long long plane;   /* ny * nz */
    long long lanes;   /* plane / v */
    long long nz;      /* input row length */
    long long ozs;     /* output row stride: nz, or nz padded to a 16-byte multiple (then v = 1) */
    int v;             /* elements per lane: 2, or 1 for an odd y-z plane or padded rows */
    int block0;        /* first block of this cube */
};

struct sf_xbargs {
    const struct sf_xcube *cubes;   /* ordered by block0 */
    int n;
    int pad_;
};

/* fused y/z filter + window statistics + threshold + mask union */
struct sf_dargs {
    const void *src[SF_MAX_SRC];
    unsigned int *mask;
    float *mean;       /* [n_filters][nwin] or null */
    float *stdv;       /* [n_filters][nwin] or null */
    int fidx[SF_MAX_SRC][SF_MAX_NZF];
    long long nx, ny, nz, nw32;
    int nwx, nwy, nwz, nwin;
    float k;
    int *err;          /* set non-zero when a bounded wait expires */
    int wid0;          /* window of block 0 (launches over a range of windows) */
    int pad_;
    long long wait_ns; /* limit of every bounded wait (%globaltimer ns) */
    long long xorg;    /* x-plane of window 0 (an x slab inside a cube with halo planes) */
};

/* Persistent batched kernel: a unit is one cube (or one x-slab of a cube)
 * with its x pass split into items of lanes and its windows as items. */
struct sf_unit {
    struct sf_dargs args;       /* the cube's window-kernel arguments */
    const void *xsrc;           /* x-pass input (the cube) */
    void *xdst[SF_MAX_XOUT];    /* x-pass outputs (scratch slots of this cube) */
    long long x0, x1;           /* x-planes of this unit (multiples of wx) */
    long long plane;            /* ny * nz */
    long long lanes;            /* plane / xv */
    int xv;                     /* elements per x lane: 1 or 2 */
    int tma;                    /* slabs by TMA (1) or cp.async (0) */
    int map_base;               /* first tensor map of this unit */
    int n_xitems;               /* x items of this unit */
    int wx0;                    /* first window-grid x of this unit */
    int xlanes;                 /* lanes per x item */
};

struct sf_item {
    int unit;
    int kind;                   /* 0: x lanes, 1: window */
    int index;                  /* x item or window of the unit */
    int pad_;
};

struct sf_pargs {
    const struct sf_unit *units;
    const struct sf_item *items;
    const void *maps;           /* 64-byte aligned tensor maps */
    int *head;                  /* next item (reset to 0 before each launch) */
    int *xdone;                 /* per unit: x items completed (reset to 0) */
    int *err;
    int n_items;
    int xextra;                 /* test hook: x items a window waits for beyond its unit's */
    long long wait_ns;          /* limit of every bounded wait (%globaltimer ns) */
};

/* y/z filter of one filter, writing float32 filtered values */
struct sf_fargs {
    const void *src;
    float *out;
    long long nx, ny, nz;
};

#endif
