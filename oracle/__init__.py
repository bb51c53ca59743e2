"""FP64 CPU oracle of the SurfelWarp per-frame hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA library never links, imports or calls it,
and it shares no code with the CUDA path.

The oracle is a plain, slow, step-by-step restatement of the method in the
paper's order and notation (SurfelWarp, Gao & Tedrake 2019):

* ``dq``        -- quaternion / dual-quaternion algebra (Sec. 3, Eq. 1-3)
* ``depth``     -- depth image processing (Sec. 5, Eq. 4)
* ``skinning``  -- k-NN skinning and the node graph (Sec. 6.5, Eq. 1)
* ``solver``    -- association, residuals, Jacobians, JtJ, block-Jacobi PCG,
                   Gauss-Newton (Sec. 7, Eq. 9-11; Sec. 8)
* ``fusion``    -- index map, live-frame fusion, inverse warp (Sec. 6.1,
                   Eq. 5-6; Sec. 4, Eq. 3)
* ``rigid``     -- rigid pre-alignment before the non-rigid solve (Sec. 7)
* ``visibility`` -- opaque splat visibility before the solve (Sec. 7)
* ``append``    -- live skinning, compressive test, appending and removal
                   (Sec. 6.2-6.4, Eq. 7-8)
* ``stream``    -- the five per-stream calls over host memory

Floating point is FP64 throughout, except where a floating-point result
decides an integer (k-NN selection, projective association, index-map
sub-pixel and depth key, fusion candidate tests): those decisions are taken in
FP32 with a fixed operation order, the precision the CUDA kernels take them in.

Readings of passages the paper leaves open are restated next to the code
that implements them.  Parity unpinned: the
paper-faithfulness of those readings (thresholds, node radius, association
method, parameterisation); they are decisions, not facts the paper fixes.
"""
from . import dq, depth, skinning, solver, fusion, rigid, visibility, append, stream  # noqa: F401
from .stream import OracleStream, Params  # noqa: F401
