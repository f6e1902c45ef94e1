"""Dense matrices built directly from the definitions, for pinning the oracle.

Pure-Python loops over indices (tiny images only). Nothing here is shared with
the oracle: the Toeplitz, Kronecker and difference matrices are written out
entry by entry from their definitions.
"""
import numpy as np


def toeplitz_dense(length, taps):
    """T[i, i'] = taps[(i' - i) + r] for |i' - i| <= r (zero boundary)."""
    r = (len(taps) - 1) // 2
    T = np.zeros((length, length))
    for i in range(length):
        for ip in range(length):
            a = ip - i
            if -r <= a <= r:
                T[i, ip] = taps[a + r]
    return T


def blur_dense(height, width, taps):
    """H with (H x)[i*w+j] = sum_{a,b} g_a g_b x[(i+a)*w + (j+b)] (in-image only)."""
    n = height * width
    r = (len(taps) - 1) // 2
    H = np.zeros((n, n))
    for i in range(height):
        for j in range(width):
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < height and 0 <= jj < width:
                        H[i * width + j, ii * width + jj] += taps[a + r] * taps[b + r]
    return H


def grad_dense(height, width):
    """L = [D_x; D_y]: (D_x x)(i,j) = x(i,j+1) - x(i,j) for j < w-1, zero row at j = w-1;
    (D_y x)(i,j) = x(i+1,j) - x(i,j) for i < h-1, zero row at i = h-1."""
    n = height * width
    L = np.zeros((2 * n, n))
    for i in range(height):
        for j in range(width):
            row = i * width + j
            if j < width - 1:
                L[row, i * width + j + 1] = 1.0
                L[row, i * width + j] = -1.0
            if i < height - 1:
                L[n + row, (i + 1) * width + j] = 1.0
                L[n + row, i * width + j] = -1.0
    return L


def operator_dense(height, width, taps, w, gamma):
    H = blur_dense(height, width, taps)
    L = grad_dense(height, width)
    A = H.T @ H
    E = L.T @ np.diag(w) @ L
    return A, E, A + gamma * E
