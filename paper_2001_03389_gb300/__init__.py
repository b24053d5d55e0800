"""GB300-native RFI mitigation: time- and frequency-domain sigma cuts."""
