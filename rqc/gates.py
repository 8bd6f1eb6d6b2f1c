"""Gate set of Sycamore-style random quantum circuits (SM Sec. I).

The three single-qubit gates are the square roots of X, Y and
W = (X + Y)/sqrt(2), each written with the global phase the paper prints
for it.  The two-qubit gate is the five-parameter fSim gate.  The paper's
printed fSim matrix repeats exp(i(D+ + D-)) cos(theta) on both middle
diagonal entries; with every Delta set to zero (the setting used here) that
detail has no effect, and the matrix reduces to

    [[1, 0,            0,            0          ],
     [0, cos t,        -i sin t,     0          ],
     [0, -i sin t,     cos t,        0          ],
     [0, 0,            0,            exp(-i phi)]]

Basis order of a two-qubit matrix: |q_a q_b> with the lower qubit id a as
the most significant bit (row/column index = 2*b_a + b_b).
"""

import numpy as np

_H = np.sqrt(2.0) / 2.0

SQRT_X = _H * np.array([[1.0, -1.0j], [-1.0j, 1.0]], dtype=np.complex128)
SQRT_Y = _H * np.array([[1.0, -1.0], [1.0, 1.0]], dtype=np.complex128)
SQRT_W = _H * np.array(
    [[1.0, -_H * (1.0 + 1.0j)], [_H * (1.0 - 1.0j), 1.0]], dtype=np.complex128
)

SINGLE_QUBIT_GATES = (SQRT_X, SQRT_Y, SQRT_W)
SINGLE_QUBIT_NAMES = ("sqrtX", "sqrtY", "sqrtW")


def fsim(theta=np.pi / 2, phi=np.pi / 6, d_plus=0.0, d_minus=0.0, d_minus_off=0.0):
    """Five-parameter fSim gate (SM Sec. I).  The middle block uses
    exp(i(D+ + D-)) on the (01,01) entry and exp(i(D+ - D-)) on the (10,10)
    entry, the usual reading of the printed matrix; at D = 0 both are 1."""
    c, s = np.cos(theta), np.sin(theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[1, 1] = np.exp(1j * (d_plus + d_minus)) * c
    m[1, 2] = -1j * np.exp(1j * (d_plus - d_minus_off)) * s
    m[2, 1] = -1j * np.exp(1j * (d_plus + d_minus_off)) * s
    m[2, 2] = np.exp(1j * (d_plus - d_minus)) * c
    m[3, 3] = np.exp(1j * (2.0 * d_plus - phi))
    return m
