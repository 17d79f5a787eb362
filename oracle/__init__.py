"""CPU oracle for the Cordic-based Loeffler DCT image codec.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It is a plain, slow, obviously correct
restatement of what the GPU library computes and shares no code with it:

* ``exact_dct``      FP64 textbook DCT-II / IDCT (Eq. 3, 4, 6, 7) and the
                     exact-DCT compression pipeline (the "DCT" rows of
                     Tables 3 and 4).
* ``cordic_loeffler`` the fixed-point Cordic-based Loeffler 8-point forward
                     and inverse flow graphs (Sec. 2.5.2, Fig. 1), written
                     generically so the same code runs on integers and on
                     intervals.
* ``codec``          plane-level pipeline: padding, level shift, 2-D
                     transform, quantiser, dequantiser, inverse, descale
                     (Sec. 3.2: DCT, quantiser and IDCT as separate steps).
* ``psnr``           SSE and PSNR (Eq. 23, 24).
* ``ijg``            JPEG base tables and the IJG quality scaling.
* ``interval``       interval propagation through every node of both flow
                     graphs, proving the int32 word width is enough.
* ``mlp``, ``features``, ``ratecontrol``  the learned rate controller's
                     network (FP64), its 80 inputs and the 8-step bisection.

Parity status: the exact DCT, the fixed-point codec, SSE/PSNR, the IJG
tables, the features, the MLP and the bisection are pinned by the tests in
``tests/test_oracle_*.py``.  The PSNR values printed in Tables 3 and 4 are
parity unpinned: the images and the quality setting behind them are not
available.
"""
