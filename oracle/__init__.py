"""CPU oracle for multiple-amplitude tensor network contraction.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or
executes anything here; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares no
code with the CUDA library and takes its inputs from the seeded generators
in ``rqc`` only.

Contents (all complex128 / float64):

* ``sv``     -- state-vector simulator in plain C: amp_b = <b|U|0^n> (SM Sec. II).
* ``brute``  -- the full 2^n x 2^n circuit unitary from per-gate matrices,
                for n <= 10 (an independent check of ``sv``).
* ``tn``     -- an independent pairwise tensor-network contractor over the
                *unfused* network (|0> vectors, 2x2 and 4x4 gates, output
                projections), with first-level slicing as a sum over fixed
                wire values (SM Sec. IV.B) and a dynamic memo cache over
                shared sub-networks.
* ``xeb``    -- linear cross-entropy benchmarking fidelity and the
                Porter-Thomas law of Eq. (fxeb).
* ``mlp``    -- forward/backward of the 2x128 MLP cost model in float64.
"""
