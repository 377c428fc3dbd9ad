"""FP64 CPU oracle of the Zak-OTFS receiver hot path (SS-CGA).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's receiver in NumPy float64 / complex128.  It exists to
check the CUDA library, never to stand in for it: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` leg of
``bench.py`` may import it.  It shares no code with ``paper_2604_02266_gb300``
(no kernels, tables, constants or helpers) and neither side imports the other.

Modules, each citing the passage it follows:

* :mod:`oracle.zak`        -- discrete Zak transform pair (Sec. III-B, Eq. iZak, Eq. zak)
* :mod:`oracle.ddchannel`  -- point-pilot read-off (Eq. heff, Eq. heff_exp/heff_hadamard),
  dominant-path thresholding (Eq. heff_thres), dense channel matrix (Eq. Hdd),
  structured-sparse index maps and phases (Eq. map_chMatDD_col, Eq. herm_mapping,
  Sec. IV-B "Phase correction"), integer-offset time-domain channel (Eq. y_discrete_td)
* :mod:`oracle.equalizer`  -- SS forward/Hermitian MVMs (Eq. sparse_mvm, Eq. sparse_herm_mvm),
  compute-aware CGA (Algorithm 1), direct LMMSE by Cholesky (Eq. lmmse), MIMO stacking
* :mod:`oracle.qam`        -- Gray square QAM, hard demodulation (Eq. demod), max-log LLRs
* :mod:`oracle.receiver`   -- the receiver stages composed per frame, as the GPU batch runs them
* :mod:`oracle.mrc`        -- SS-MRC, the maximal-ratio-combining decision-feedback equaliser
  (Sec. III-B "Equalization", MRC paragraph), in the delay-time domain

Every function whose result is not pinned by a test against something other than
itself says "parity unpinned" in its docstring; at present there is none.
"""

from . import zak, ddchannel, equalizer, qam, receiver, mrc  # noqa: F401
